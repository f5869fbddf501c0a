"""Pins of the oracle's histogram reading of coexistence densities
(config 2's measurement: Sec. II E's coexistence densities from the density
histogram of a separated state; 2048 bins on [0, 3), the two highest peaks on
either side of the critical density 1, each refined to the mean of the
densities within +-2 bins).  The samples are synthetic with known answers."""
import numpy as np

from oracle import analysis as A

NB, LO, HI = 2048, 0.0, 3.0
W = (HI - LO) / NB
EDGES = np.linspace(LO, HI, NB + 1)
CENTRES = 0.5 * (EDGES[:-1] + EDGES[1:])


def population(pk, parts):
    """Values at bin centres pk + offset, `count` of each: [(offset, count), ...]."""
    return np.concatenate([np.full(n, CENTRES[pk + o]) for o, n in parts])


def test_peak_bins_and_refined_means_are_exact():
    """Two populations at known bins.  Inside the +-2-bin window each is
    asymmetric (so a narrower window changes the mean); just outside it sit
    extra values (so a wider window changes it too).  A flat background of one
    value per bin between the peaks makes no peak of its own."""
    iv, il = 300, 1100                     # rho_V ~ 0.44, rho_L ~ 1.61
    vin = population(iv, [(0, 600), (-1, 200), (1, 250), (2, 120), (-2, 40)])
    vout = population(iv, [(3, 80), (-3, 30)])
    lin = population(il, [(0, 900), (-2, 310), (-1, 100), (1, 90), (2, 15)])
    lout = population(il, [(-3, 200), (4, 60)])
    bg = CENTRES[iv + 6:il - 6]
    rho = np.concatenate([vin, vout, lin, lout, bg])
    counts, _ = np.histogram(rho, bins=NB, range=(LO, HI))
    # the bin centres alone (no raw values)
    rl0, rv0 = A.coexistence_from_histogram(counts, LO, HI)
    assert rl0 == CENTRES[il] and rv0 == CENTRES[iv]
    # refined: the mean of the values inside the +-2-bin windows
    rl, rv = A.coexistence_from_histogram(counts, LO, HI, rho_values=rho)
    assert abs(rv - vin.mean()) < 1e-14 and abs(rl - lin.mean()) < 1e-14
    # the extra values outside the windows would have moved both means
    assert abs(np.concatenate([vin, vout]).mean() - vin.mean()) > 1e-4
    assert abs(np.concatenate([lin, lout]).mean() - lin.mean()) > 1e-4


def test_separated_state_like_sample():
    """A sample shaped like a separated spinodal state: two narrow bulk
    populations (spread 3e-4, below a bin width) of unequal size around known
    means and a uniform interface population between them; the estimates are
    the bulk means to well within the 1e-4 bar that the FP32-vs-FP64
    coexistence gate uses."""
    rng = np.random.default_rng(2)
    mv, ml = 0.4257, 1.6573              # Maxwell at T = 0.9 to 4 digits
    vap = mv + 3e-4 * rng.standard_normal(150_000)
    liq = ml + 3e-4 * rng.standard_normal(350_000)
    iface = rng.uniform(mv, ml, 40_000)
    rho = rng.permutation(np.concatenate([vap, liq, iface]))
    counts, _ = np.histogram(rho, bins=NB, range=(LO, HI))
    rl, rv = A.coexistence_from_histogram(counts, LO, HI, rho_values=rho)
    assert abs(rv - vap.mean()) < 1e-5 and abs(rl - liq.mean()) < 1e-5
    assert abs(rv - mv) < 1e-5 and abs(rl - ml) < 1e-5
    # the order of the result: (rho_L, rho_V)
    assert rl > 1.0 > rv


def test_split_decides_the_sides():
    """A liquid peak higher than the vapour peak, and a vapour peak higher than
    the liquid one: each side's own maximum is taken."""
    for nv, nl in ((1000, 5000), (5000, 1000)):
        rho = np.concatenate([np.full(nv, CENTRES[200]), np.full(nl, CENTRES[1200])])
        counts, _ = np.histogram(rho, bins=NB, range=(LO, HI))
        rl, rv = A.coexistence_from_histogram(counts, LO, HI, rho_values=rho)
        assert rv == CENTRES[200] and rl == CENTRES[1200]


def test_smoothed_peak_moves_continuously():
    """A state still separating has a broad, nearly flat-topped bulk peak: here
    a liquid population spread uniformly over six bins around ml.  Shifting
    every value by a fraction of a bin shifts the smoothed-peak estimate by
    that fraction (the window is centred on a peak that moves continuously);
    the highest-bin reading jumps by whole bins instead, which is why two
    slightly different runs (FP32 and FP64 of a chaotic separation) can
    differ there by a bin width (1.5e-3 at 2048 bins on [0, 3))."""
    rng = np.random.default_rng(3)
    ml, mv = CENTRES[1100], CENTRES[300]
    liq = ml + W * rng.uniform(-3.0, 3.0, 400_000)
    vap = mv + 3e-4 * rng.standard_normal(100_000)
    iface = rng.uniform(mv, ml, 20_000)
    jumps = []
    for d in (0.0, 0.2, 0.45, 0.7, 0.95):
        rho = np.concatenate([vap, liq + d * W, iface])
        counts, _ = np.histogram(rho, bins=NB, range=(LO, HI))
        rl, rv = A.coexistence_from_histogram(counts, LO, HI, rho_values=rho, peak="smoothed",
                                              halfwidth=4)
        assert abs(rl - (ml + d * W)) < 0.1 * W, (d, (rl - ml) / W)
        assert abs(rv - vap.mean()) < 1e-5
        rb, _ = A.coexistence_from_histogram(counts, LO, HI, rho_values=rho)
        jumps.append((rb - (ml + d * W)) / W)
    print("\nhighest-bin reading minus the true centre, in bins:", np.round(jumps, 2))


def test_smoothed_peak_on_a_separated_sample():
    """On narrow bulk populations the smoothed reading equals the bulk means,
    as the highest-bin reading does."""
    rng = np.random.default_rng(2)
    mv, ml = 0.4257, 1.6573
    vap = mv + 3e-4 * rng.standard_normal(150_000)
    liq = ml + 3e-4 * rng.standard_normal(350_000)
    iface = rng.uniform(mv, ml, 40_000)
    rho = rng.permutation(np.concatenate([vap, liq, iface]))
    counts, _ = np.histogram(rho, bins=NB, range=(LO, HI))
    for hw in (2, 4):
        rl, rv = A.coexistence_from_histogram(counts, LO, HI, rho_values=rho, peak="smoothed",
                                              halfwidth=hw)
        assert abs(rv - vap.mean()) < 1e-5 and abs(rl - liq.mean()) < 1e-5
