"""Sec. III bubble experiments on the CUDA path: surface tension of a planar
interface, the critical radius of Eq. (raggio_c) and bubble growth against the
Rayleigh-Plesset equation (Eq. rp)."""
import json
import os

import numpy as np
import pytest

from tests.conftest import has_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_planar_interface_surface_tension():
    """Sec. III A: sigma of the relaxed planar interface at T = 0.8, kappa = 1e-4,
    ds = 1/256, tau = 1e-3 (the paper: 4.8747e-3; measured +0.07 %), with the
    liquid plateau on the Maxwell density and the vapour plateau 1 % below it.
    FP32 shifted storage (its coexistence matches FP64 to 1e-6)."""
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import eos
    from paper_1802_01272_gb300 import experiments as X
    sigma, prof = X.planar_interface_sigma(precision=P.LBM_FP32_SHIFTED)
    want = GOLD["surface_tension_T0.8_kappa1e-4"]["ds_1_256"]
    rl, rv = eos.coexistence(0.8)
    print(f"\nsigma planar = {sigma:.6e} paper {want:.6e} rel {(sigma - want) / want:+.2e}; "
          f"rho_L {prof.max():.6f} ({rl:.6f}) rho_V {prof.min():.6f} ({rv:.6f})")
    assert abs(sigma - want) / want < 5e-3
    assert abs(prof.max() - rl) / rl < 1e-3 and abs(prof.min() - rv) / rv < 2e-2


def test_phase_diagram_vapour_density_against_maxwell():
    """Sec. II E: planar-interface coexistence densities on the paper's grid
    (CTU2, tau = 1e-3, dt = 1e-4, ds = 1/256) stay close to Maxwell's from
    T = 0.7 up, while at T = 0.6 the vapour density sits about 8 % under it
    (measured: -3.2 % at T = 0.7, -1.0 % at 0.8, -10.2 % at 0.6)."""
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import eos
    from paper_1802_01272_gb300 import experiments as X
    g = GOLD["phase_diagram_vapour_deviation"]
    dev = {}
    for T in (g["T_low"], g["T_good_agreement_min"], 0.8):
        _, prof = X.planar_interface_sigma(T=T, Lx=128, t_end=20.0, precision=P.LBM_FP32_SHIFTED)
        rl, rv = eos.coexistence(T)
        pl, pv = X.slab_plateaus(prof)
        dev[T] = (pl / rl - 1.0, pv / rv - 1.0)
        print(f"\nT={T}: rho_L {dev[T][0]:+.3e} rho_V {dev[T][1]:+.3e} of Maxwell")
    for T in (g["T_good_agreement_min"], 0.8):
        assert abs(dev[T][0]) < 2e-3 and abs(dev[T][1]) < 0.05
    low = -dev[g["T_low"]][1]
    assert abs(low - g["vapour_rel_diff_at_T_low"]) < 0.04 and abs(dev[g["T_low"]][0]) < 2e-3
    assert low > -dev[g["T_good_agreement_min"]][1] > -dev[0.8][1] > 0


def test_lattice_spacing_dependence_of_sigma_and_coexistence():
    """Sec. III A gives sigma for ds = 1/128 (4.8754e-3) as well as 1/256, the
    two nearly equal; Sec. II E has the coexistence densities approach
    Maxwell's as ds falls.  Measured (T = 0.8, tau = 1e-3): sigma 4.841e-3
    at ds = 1/128 (-0.7 %), vapour -3.9 % at 1/128 against -1.0 % at 1/256."""
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import eos
    from paper_1802_01272_gb300 import experiments as X
    want = GOLD["surface_tension_T0.8_kappa1e-4"]
    _, rv = eos.coexistence(0.8)
    out = {}
    for key, ds, Lx in (("ds_1_128", 1 / 128, 256), ("ds_1_256", 1 / 256, 512)):
        sigma, prof = X.planar_interface_sigma(ds=ds, Lx=Lx, precision=P.LBM_FP32_SHIFTED)
        out[key] = (sigma, abs(prof.min() - rv) / rv)
        print(f"\n{key}: sigma {sigma:.6e} (paper {want[key]:.6e}, rel {(sigma - want[key]) / want[key]:+.2e}) "
              f"rho_V rel {out[key][1]:.3e}")
        assert abs(sigma - want[key]) / want[key] < 1e-2
    assert out["ds_1_256"][1] < out["ds_1_128"][1]


def test_coexistence_approaches_maxwell_as_tau_decreases():
    """Sec. II E (dependence of rho_L, rho_V on tau at T = 0.8): the planar
    interface's vapour density moves toward the Maxwell value as tau falls."""
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import eos
    from paper_1802_01272_gb300 import experiments as X
    _, rv = eos.coexistence(0.8)
    dev = []
    for tau in (1e-2, 1e-3):
        _, prof = X.planar_interface_sigma(tau=tau, t_end=30.0, precision=P.LBM_FP32_SHIFTED)
        dev.append(abs(prof.min() - rv) / rv)
        print(f"\ntau={tau}: rho_V {prof.min():.6f} (Maxwell {rv:.6f}) rel {dev[-1]:.3e}")
    assert dev[1] < dev[0]


def test_critical_radius_matches_the_paper():
    """Sec. III A: with the liquid held at rho_ext = 1.923 (T = 0.8, L = 1024,
    ds = 1/256), the paper's lattice gives R_c = 76.5 ds (Eq. raggio_c: 75.7).
    A bubble seeded 1.5 nodes under it collapses and one 1.5 nodes over it
    grows."""
    from paper_1802_01272_gb300 import eos
    from paper_1802_01272_gb300 import experiments as X
    rc = GOLD["critical_radius_rho_ext_1.923"]["Rc_over_ds"]
    pred = X.critical_radius(0.8, 1.923, eos.interface_tension(0.8, 1e-4)) * 256
    print(f"\nR_c paper lattice {rc} nodes, Eq. raggio_c {pred:.2f} nodes")
    small = X.bubble_in_reservoir(rc - 1.5, 1.923, t_end=8.0, every=0.5)
    large = X.bubble_in_reservoir(rc + 1.5, 1.923, t_end=8.0, every=0.5)
    print("small R(t) nodes", np.round(small.R * 256, 2))
    print("large R(t) nodes", np.round(large.R * 256, 2))
    i = int(np.searchsorted(small.t, 1.0))
    assert small.R[-1] * 256 < small.R[i] * 256 - 3.0
    assert large.R[-1] * 256 > large.R[i] * 256 + 1.5


def test_laplace_law_for_near_critical_bubbles():
    """Laplace's law in 2D, p_B - p_inf = sigma / R (Sec. III A: the critical
    bubble of Eq. raggio_c is the one in Laplace balance with the reservoir;
    Sec. III B reads p_B and p_inf from the EOS at the bubble's centre and far
    field).  For three reservoir densities the bubble is seeded at Eq.
    raggio_c's critical radius (about 76, 58 and 42 nodes at rho_ext = 1.923,
    1.920, 1.915; T = 0.8, 1024^2, tau = 1e-3); once its interface has relaxed
    it sits in near-equilibrium (it changes by less than 1.5 nodes over the
    window).  The pressure jump, p^w(rho_centre) - p^w(rho_ring) against the
    equivalent radius of the bubble sites, falls on a straight line in 1/R
    whose slope is sigma (kappa int rho'^2 dx with the Maxwell densities).
    The line's intercept is the lattice's thermodynamic offset: its vapour
    branch lies about 1 % under Maxwell's at T = 0.8 (the planar interface
    shows the same), and at rho_V ~ 0.24 that moves p^w by ~6 % of sigma/R at
    R = 76 nodes, nearly the same for the three bubbles, so the intercept
    carries it and the slope is the check of Laplace's law."""
    from paper_1802_01272_gb300 import eos
    from paper_1802_01272_gb300 import experiments as X
    T, ds = 0.8, 1 / 256
    sigma = eos.interface_tension(T, 1e-4)
    inv_r, dps = [], []
    for rho_ext in (1.923, 1.920, 1.915):
        r0 = X.critical_radius(T, rho_ext, sigma) / ds
        run = X.bubble_in_reservoir(round(r0), rho_ext, T=T, t_end=3.0, every=0.1)
        win = (run.t >= 1.5 - 1e-12) & (run.t <= 3.0 + 1e-12)
        R = run.R[win]
        dp = eos.pressure(run.rho_center[win], T) - eos.pressure(run.rho_inf[win], T)
        drift = abs(R[-1] - R[0]) / ds
        inv_r.append(1.0 / R.mean())
        dps.append(dp.mean())
        print(f"\nrho_ext {rho_ext}: seed {round(r0)} nodes, R {R.mean() / ds:.2f} nodes, "
              f"dp {dp.mean():.5e}, dp R / sigma {dp.mean() * R.mean() / sigma:.4f}, "
              f"drift {drift:.2f} nodes")
        assert drift < 1.5
    slope, icpt = np.polyfit(inv_r, dps, 1)
    print(f"fit: slope {slope:.5e} (sigma {sigma:.5e}, ratio {slope / sigma:.4f}), "
          f"intercept {icpt:.3e} ({icpt / (sigma * max(inv_r)):+.3f} of the largest sigma/R)")
    assert abs(slope / sigma - 1.0) < 0.05
    assert abs(icpt) < 0.15 * sigma * max(inv_r)


def test_rayleigh_plesset_growth():
    """Sec. III B: a supercritical bubble (rho_ext = 1.923) grows as Eq. (rp)
    predicts from the pressures measured at its centre and at r_inf = R_BC,
    starting from the lattice state after the interface has relaxed (t = 2);
    2048^2 nodes, so that r_inf / R stays large (the paper notes RP holds only
    while that ratio is large).  Measured: RP ends 2 % of the growth away
    from the lattice radius."""
    from paper_1802_01272_gb300 import experiments as X
    run = X.bubble_in_reservoir(110, 1.923, L=2048, t_end=8.0, every=0.1)
    t, R = X.rp_prediction(run, 2.0)
    lb = run.R[np.searchsorted(run.t, t[0] - 1e-12):]
    print("\nt", np.round(t[::10], 2))
    print("R_LB nodes", np.round(lb[::10] * 256, 2))
    print("R_RP nodes", np.round(R[::10] * 256, 2))
    growth = lb[-1] - lb[0]
    assert growth * 256 > 3.0
    assert abs(R[-1] - lb[-1]) < 0.1 * growth


def test_sheared_bubble_deformation_and_tilt():
    """Sec. III C: a bubble growing in sheared superheated liquid (1024 x 512,
    walls, rho_ext = 1.90, tau = 1e-2) deforms linearly with the capillary
    number of its current size for Ca <= 0.2 (the paper fits D = 0.89 Ca,
    Taylor's steady value is 1.02 Ca; measured here 0.854, bar 0.06; on the
    paper's 6144^2 lattice at its shear rates the joint slope is 0.95, see
    test_gpu_configs), tilts at ~pi/4 to the flow at first and less as it
    grows, less at the higher shear rate, and grows at a rate that does not
    depend on the shear."""
    from paper_1802_01272_gb300 import experiments as X
    gold = GOLD["shear_deformation_T0.8"]
    lo = X.sheared_bubble(40, 0.05, t_end=10.0, every=1.0)
    hi = X.sheared_bubble(40, 0.15, t_end=10.0, every=1.0)
    for r in (lo, hi):
        print(f"\ngamma_dot {r.shear_rate:.4f}: R nodes {np.round(r.R * 256, 1)}")
        print(f"  D/Ca {np.round(r.D / np.maximum(r.Ca, 1e-9), 3)}  theta {np.round(r.theta, 3)}")
    sel = (lo.t >= 3.0) & (lo.Ca <= 0.2)
    slope = float(np.sum(lo.D[sel] * lo.Ca[sel]) / np.sum(lo.Ca[sel] ** 2))
    print(f"  D = {slope:.3f} Ca (paper {gold['D_over_Ca_fit']}, Taylor {gold['D_over_Ca_taylor']})")
    assert abs(slope - gold["D_over_Ca_fit"]) < 0.06   # measured 0.854
    assert abs(lo.theta[1] - np.pi / 4) < 0.1 and abs(hi.theta[1] - np.pi / 4) < 0.15
    assert lo.theta[-1] < lo.theta[2] and hi.theta[-1] < lo.theta[-1]
    assert lo.R[-1] > 2.5 * lo.R[0]
    assert abs(hi.R[-1] - lo.R[-1]) / lo.R[-1] < 0.1


def test_config3_quiescent_bubble_grows_in_superheated_liquid():
    """Config 3 of the quiescent-growth experiments (Sec. III B at T = 0.9):
    a tanh seed of radius 20 nodes at the Maxwell vapour density in liquid
    held at rho_ext = 1.58 (Eq. raggio_c: R_c = 11.8 nodes) grows without
    stopping, and the reservoir keeps the far field at rho_ext.  2048^2
    nodes, tau = 1e-3, t = 3 (30000 steps)."""
    from paper_1802_01272_gb300 import eos
    from paper_1802_01272_gb300 import experiments as X
    rc = X.critical_radius(0.9, 1.58, eos.interface_tension(0.9, 1e-4)) * 256
    assert rc < 15.0
    run = X.bubble_in_reservoir(20, 1.58, T=0.9, L=2048, tau=1e-3, t_end=3.0, every=0.5)
    print("\nR nodes", np.round(run.R * 256, 2), " rho_inf", np.round(run.rho_inf, 4))
    assert np.all(np.diff(run.R[1:]) > 0) and run.R[-1] > 3.5 * run.R[0]
    assert np.abs(run.rho_inf - 1.58).max() < 2e-3
