"""Host-side pieces of the bubble experiments (no GPU): the library's
Eq. (raggio_c) and Rayleigh-Plesset integrator against the oracle's closed
forms, which the oracle pins hold to the paper's printed numbers."""
import math

import numpy as np


def test_free_energy_and_critical_radius_agree_with_oracle():
    from oracle import analysis as A
    from paper_1802_01272_gb300 import experiments as X
    for rho in (0.2, 1.0, 1.9):
        assert abs(X.free_energy(rho, 0.8) - A.psi(rho, 0.8)) < 1e-14
    for rho_ext in (1.87, 1.9, 1.923):
        got = X.critical_radius(0.8, rho_ext, 4.8747e-3)
        want = A.critical_radius(4.8747e-3, rho_ext, 0.8)
        assert abs(got - want) / want < 1e-9
    # Sec. III B: R_c rises with rho_ext (inset of the critical-radius figure)
    r = [X.critical_radius(0.8, e, 4.8747e-3) for e in (1.87, 1.9, 1.923)]
    assert r[0] < r[1] < r[2]


def test_rayleigh_plesset_agrees_with_oracle_rk4():
    from oracle import analysis as A
    from paper_1802_01272_gb300 import experiments as X
    kw = dict(r_inf=1.5, sigma=4.87e-3, rho_l=1.93, mu_l=1.93 * 0.8 * 1e-3)
    pb = lambda t: 0.1 + 0.002 * t                       # noqa: E731
    pf = lambda t: 0.08                                  # noqa: E731
    times = np.array([0.0, 0.5, 1.0, 2.0])
    R = X.rayleigh_plesset(0.35, 0.01, times, pb, pf, **kw)
    t, Ro, _ = A.rp_integrate(0.35, 0.01, 2.0, 1e-3, p_b=pb, p_inf=pf, **kw)
    for te, r in zip(times, R):
        assert abs(r - np.interp(te, t, Ro)) < 1e-10
    # Laplace balance: a bubble with p_B - p_inf = sigma / R stays put
    R = X.rayleigh_plesset(0.3, 0.0, times, lambda t: 0.08 + 4.87e-3 / 0.3, pf, **kw)
    assert np.abs(R - 0.3).max() < 1e-13


def test_bubble_fields_geometry():
    from paper_1802_01272_gb300 import experiments as X
    rho, ux, uy = X.bubble_fields(128, 96, 20.0, 0.24, 1.9, 1.0)
    assert rho.shape == (96, 128) and not ux.any() and not uy.any()
    assert abs(rho[48, 64] - 0.24) < 1e-9 and abs(rho[0, 0] - 1.9) < 1e-9
    nb = (rho < 0.5 * (0.24 + 1.9)).sum()
    assert abs(math.sqrt(nb / math.pi) - 20.0) < 0.5


def test_critical_radius_bisection_logic():
    """Sec. III A's estimate R_c = (R_g + R_s)/2 with R_g = R_s + 1 node, on a
    stand-in classifier (the GPU run is replaced by a threshold at 76.3)."""
    import pytest
    from paper_1802_01272_gb300 import experiments as X
    calls = []

    def fate(r):
        calls.append(r)
        return 1 if r > 76.3 else -1
    rs, rg, rc, seen = X.critical_radius_bisection(1.923, 60, 100, fate=fate)
    assert (rs, rg, rc) == (76, 77, 76.5)
    assert len(calls) <= 2 + 6 and seen[76] == -1 and seen[77] == 1
    with pytest.raises(ValueError):
        X.critical_radius_bisection(1.923, 80, 100, fate=fate)     # 80 grows
    with pytest.raises(ValueError):
        X.critical_radius_bisection(1.923, 60, 100, fate=lambda r: 0 if r == 80 else fate(r))


def test_bubble_fate_reads_growth_after_relaxation():
    from paper_1802_01272_gb300 import experiments as X
    from paper_1802_01272_gb300.binding import Params
    t = np.arange(0.0, 8.01, 0.5)
    p = Params(Lx=64, Ly=64, ds=1 / 256)
    mk = lambda R: X.BubbleRun(t=t, R=np.asarray(R) / 256, rho_center=t * 0, rho_inf=t * 0,  # noqa: E731
                               r_inf=1.0, params=p)
    dip = np.where(t < 1.0, 80 - 5 * t, 75 + 0.5 * (t - 1.0))   # relaxes down, then grows
    assert X.bubble_fate(mk(dip)) == 1
    assert X.bubble_fate(mk(80 - 0.9 * t)) == -1
    assert X.bubble_fate(mk(80 + 0.01 * t)) == 0


def test_phase_diagram_driver_plumbing(monkeypatch):
    """phase_diagram runs one planar interface per temperature with the given
    grid and pairs its plateaus with the Maxwell densities (the lattice run
    itself is replaced by a stand-in profile here; the GPU tests run it)."""
    from paper_1802_01272_gb300 import eos
    from paper_1802_01272_gb300 import experiments as X
    seen = []

    def fake(T, kappa, ds, Lx, tau, t_end, precision, stream):
        seen.append((T, kappa, ds, Lx, tau, t_end))
        rl, rv = eos.coexistence(T)
        return 1e-3 * T, np.array([rv * 0.9, rl, rv * 0.9])
    monkeypatch.setattr(X, "planar_interface_sigma", fake)
    rows = X.phase_diagram((0.6, 0.8), Lx=96, t_end=5.0)
    assert [r["T"] for r in rows] == [0.6, 0.8]
    assert seen == [(0.6, 1e-4, 1 / 256, 96, 1e-3, 5.0), (0.8, 1e-4, 1 / 256, 96, 1e-3, 5.0)]
    for r in rows:
        rl, rv = eos.coexistence(r["T"])
        assert r["maxwell_L"] == rl and r["maxwell_V"] == rv
        assert r["rho_L"] == rl and abs(r["rho_V"] / rv - 0.9) < 1e-12
        assert r["rho_max"] == rl and r["rho_min"] == r["rho_V"]


def test_slab_plateaus_ignore_interface_overshoot():
    """The plateau reader takes medians over the bulk of each phase: an
    overshoot next to an interface (which the extremes would report) and a
    spike one node wide inside the window do not move it."""
    from paper_1802_01272_gb300 import experiments as X
    n = 128
    x = np.arange(n, dtype=np.float64)
    prof = 0.3 + 0.8 * (np.tanh((x - n / 4) / 2.0) - np.tanh((x - 3 * n / 4) / 2.0))
    prof[n // 4 + 6] += 0.05      # overshoot on the liquid side of an interface
    prof[3 * n // 4 + 6] -= 0.05  # undershoot on the vapour side
    prof[n // 2 + 1] += 0.2       # a one-node spike inside the liquid window
    pl, pv = X.slab_plateaus(prof)
    assert abs(pl - 1.9) < 1e-9 and abs(pv - 0.3) < 1e-9  # tanh tails
    assert prof.max() > 1.9 + 0.1 and prof.min() < 0.3 - 0.04
