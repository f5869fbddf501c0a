"""The benchmark configurations 2-4 at their stated sizes (Secs. II E, III B,
III C): the spinodal sweep at 1024^2 in FP64 and FP32, the quiescent
cavitating bubble at 4096^2 for 50000 steps, and the sheared bubble at
6144^2 over six shear rates.  Every figure a test measures is printed; the
asserted bars and what they rest on are stated per test."""
import math
import os

import numpy as np
import pytest

import synth
from tests.conftest import has_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]

DT, DS = 1e-4, 1.0 / 256.0


def spinodal_run(P, T, precision, L=1024, checkpoints=(1000, 20000), seed=1):
    """Spinodal decomposition from rho = 1 (1 + 1e-2 N(0,1)), u = 0 (seed 1);
    rho at each checkpoint and the 2048-bin histogram on [0, 3) at the last."""
    lp = P.Params(Lx=L, Ly=L, T=T, tau=1e-3, precision=precision, rho_ref=1.0)
    rho, ux, uy = synth.noisy_uniform(L, L, 1.0, 1e-2, seed=seed)
    out, done = {}, 0
    with P.Lattice(lp) as Lt:
        Lt.init_rho_u(rho, ux, uy)
        for c in checkpoints:
            Lt.step(c - done)
            done = c
            out[c] = Lt.moments()[0]
        hist = Lt.histogram(2048, 0.0, 3.0)
    return out, hist


def test_config2_spinodal_sweep_fp64_and_fp32():
    """Config 2: 1024^2, T = 0.70 .. 0.98, 20000 steps (t = 2), FP64 and FP32
    shifted storage from the same seeded state.  Gates: FP32 rho within 1e-5
    of FP64 after 1000 steps, and the FP32 coexistence densities within 1e-4
    of FP64's: the peaks of the histograms smoothed over two bins, each
    refined to the mean of the densities within +-4.5 bins of it.  (Spinodal
    decomposition amplifies any difference, so the FP32 and FP64 states at
    t = 2 differ in detail; at T = 0.9 the liquid peak is still broad and
    nearly flat-topped, and the highest raw bin of the two runs fell one bin
    apart, 8.6e-4 of the density, while the smoothed peaks move
    continuously.)  Both gates apply where the fluid has separated by t = 2,
    T <= 0.9; at T = 0.95 it is in mid-separation (liquid 5 % under Maxwell,
    FP32 and FP64 3e-4 apart) and at 0.98 not yet separated.  Against
    the Maxwell construction (Sec. II E) the separated liquid sits within 2 %
    at T <= 0.9 already at t = 2; the vapour is still relaxing there (its
    density overshoots Maxwell's by a few per cent at t = 2 and approaches it
    by t = 10, as the spinodal test of the validation suite shows), and close
    to the critical point the fluid has barely separated (the growth rate of
    the instability at T = 0.98 is ~2 per time unit): those deviations are
    printed, not asserted.  Measured at T = 0.7, 0.8, 0.9: FP32 - FP64
    coexistence 8.2e-5 (the vapour at T = 0.7, 0.124), 7.0e-6, 2.9e-5; liquid
    +0.02 %, +0.04 %, -1.1 % of Maxwell."""
    import paper_1802_01272_gb300 as P
    from oracle import analysis as A
    for T in (0.70, 0.80, 0.90, 0.95, 0.98):
        r64, h64 = spinodal_run(P, T, P.LBM_FP64)
        r32, h32 = spinodal_run(P, T, P.LBM_FP32_SHIFTED)
        e1000 = float(np.abs(r32[1000] - r64[1000]).max() / np.abs(r64[1000]).max())
        c64 = A.coexistence_from_histogram(h64, 0.0, 3.0, rho_values=r64[20000].ravel(),
                                           peak="smoothed", halfwidth=4)
        c32 = A.coexistence_from_histogram(h32, 0.0, 3.0, rho_values=r32[20000].ravel(),
                                           peak="smoothed", halfwidth=4)
        ml, mv = A.maxwell(T)
        dc = max(abs(a - b) / b for a, b in zip(c32, c64))
        print(f"\nT={T}: fp32-fp64 rho@1000 {e1000:.2e}; coexistence fp64 ({c64[0]:.6f}, "
              f"{c64[1]:.6f}) fp32 ({c32[0]:.6f}, {c32[1]:.6f}) rel {dc:.2e}; Maxwell "
              f"({ml:.6f}, {mv:.6f}): liquid {(c64[0] - ml) / ml:+.3e} vapour {(c64[1] - mv) / mv:+.3e}")
        assert e1000 < 1e-5
        if T <= 0.9:  # separated by t = 2 (see above)
            assert dc < 1e-4
            assert abs(c64[0] - ml) / ml < 2e-2


def test_config3_cavitation_4096_against_rayleigh_plesset():
    """Config 3: a tanh vapour seed (R = 20 nodes, width 4) at the Maxwell
    vapour density in liquid held at rho_ext = 1.58 by the reservoir (T = 0.9,
    tau = 1e-3, Eq. raggio_c: R_c = 11.8 nodes), 4096^2 nodes, 50000 steps
    (t = 5), R(t) every 500 steps.  The bubble grows monotonically and the
    reservoir holds the far field.  Eq. (rp), integrated from the lattice state
    at t = 2 with the measured pressures (Sec. III B), follows the growth to
    within a quarter of it: Eq. (rp) takes the liquid at the interface to move
    with dR/dt, which assumes rho_V << rho_L; at T = 0.9, rho_V / rho_L = 0.26
    and the prediction falls behind the lattice (at T = 0.8, where the ratio
    is 0.12, the Rayleigh-Plesset test of the experiments suite agrees to 2 %)."""
    from paper_1802_01272_gb300 import experiments as X
    run = X.bubble_in_reservoir(20, 1.58, T=0.9, L=4096, tau=1e-3, t_end=5.0, every=0.05)
    t, R = X.rp_prediction(run, 2.0)
    lb = run.R[np.searchsorted(run.t, t[0] - 1e-12):]
    growth = lb[-1] - lb[0]
    dev = (R[-1] - lb[-1]) / growth
    print("\nt   ", np.round(run.t[::20], 2))
    print("R LB", np.round(run.R[::20] / DS, 2))
    print(f"RP from t=2: R(5) {R[-1] / DS:.2f} nodes vs LB {lb[-1] / DS:.2f} "
          f"({dev:+.3f} of the growth {growth / DS:.2f} nodes)")
    assert np.all(np.diff(run.R[20:]) > 0) and run.R[-1] > 5 * run.R[0]
    assert np.abs(run.rho_inf - 1.58).max() < 2e-3
    assert abs(dev) < 0.25


def test_config4_sheared_bubble_6144_six_shear_rates():
    """Config 4: the sheared bubble at the paper's largest size (Sec. III C):
    6144^2 nodes between walls at -+u_w, tau = 1e-2, T = 0.8, a vapour bubble
    of radius 26 nodes at rho_V = 0.23967 in liquid at rho_ext = 1.90 (a sharp
    seed: the paper gives no profile, and on this lattice at tau = 1e-2 the
    26-node seed is close to critical: sharp it grows, with a tanh edge of
    width 1 or 4 nodes it dissolves), the fluid starting in the linear shear
    profile.  Six wall speeds up to u_w = 0.8 (the paper's three rates,
    gamma_dot dt = 1.67, 3.33, 5.00 e-6, are u_w = 0.2, 0.4, 0.6; the method's
    linear stability in uniform flow ends between 0.8 and 0.85 at T = 0.8:
    test_oracle_stability), 40000 steps each (t = 4; the paper ran until the bubble
    reached the walls, >= 5e5 steps, to reach Ca ~ 0.5), the bubble's area
    fraction, D, theta and Ca = mu_L gamma_dot R^ / sigma (R^ = (a + b)/2) per
    1000 steps.  Asserted: the bubble grows at every rate, its area does not
    depend on the shear (Sec. III C) to within 5 %, and once the bubble is
    resolved as deformed (D > 0.005) it tilts into the extensional quadrant
    (0 < theta < pi/2) and deforms more at the higher rate."""
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import eos
    L, T, tau, rho_ext, rho_v, R0 = 6144, 0.8, 1e-2, 1.90, 0.23967, 26.0
    rl, rv = eos.coexistence(T)
    sigma = eos.interface_tension(T, 1e-4)
    mu_l = rl * T * tau
    thr = 0.5 * (rl + rv)
    walls = (0.1, 0.2, 0.3, 0.45, 0.6, 0.8)
    final = []
    for uw in walls:
        gdot = 2.0 * uw / (L * DS)
        lp = P.Params(Lx=L, Ly=L, T=T, tau=tau, rho_ext=rho_ext, rho_ref=rho_ext,
                      boundary=P.LBM_BC_SHEAR_WALLS, shear_rate=gdot)
        rho, _, uy = synth.bubble(L, L, rho_ext, rho_v, R0, 0.0)
        ux = synth.linear_shear(L, L, uw)
        rows = []
        with P.Lattice(lp) as Lt:
            Lt.init_rho_u(rho, ux, uy)
            for i in range(41):
                if i:
                    Lt.step(1000)
                d = Lt.diagnostics(thr)
                Rm = 0.5 * (d["a"] + d["b"]) * DS
                rows.append((i * 1000, d["nb"] / (L * L), d["D"], d["theta"],
                             mu_l * gdot * Rm / sigma))
        rows = np.array(rows)
        final.append(rows[-1])
        print(f"\nu_w = {uw:.2f} (gamma_dot dt = {gdot * DT:.3e}): step, A_rel, D, theta, Ca")
        for r in rows[::5]:
            print(f"  {int(r[0]):6d} {r[1]:.4e} {r[2]:.4f} {r[3]:+.4f} {r[4]:.4f}")
        assert rows[-1, 1] > 1.1 * rows[0, 1]
        sel = rows[:, 2] > 0.005
        assert np.all((rows[sel, 3] > 0.0) & (rows[sel, 3] < math.pi / 2))
    final = np.array(final)
    assert final[:, 1].max() / final[:, 1].min() < 1.05
    Ds = final[:, 2][final[:, 2] > 0.005]
    assert len(Ds) >= 2 and np.all(np.diff(Ds) > 0), final[:, 2]


@pytest.mark.skipif(not os.environ.get("CTULBM_LONG_RUNS"),
                    reason="two 5e5-step runs at 6144^2, ~22 GPU-minutes: set CTULBM_LONG_RUNS=1")
def test_config4_long_runs_at_the_papers_shear_rates():
    """Config 4 at the paper's size and two of its shear rates (Sec. III C and
    its figures: gamma_dot dt = 1.67e-6 and 5.00e-6, u_w = 0.2 and 0.6): the
    6144^2 sheared bubble (sharp 26-node seed, tau = 1e-2) to t = 50
    (t / dt = 5e5, the time of the paper's density plots), the shape every 0.5.
    The paper prints Ca = 0.18 and 0.61 at that time; D grows linearly with Ca
    up to ~0.2 (best fit D = 0.89 Ca over its three rates); the lower rate
    keeps the higher tilt.  Measured: Ca(t = 50) = 0.169 and 0.562 (R = 822
    and 910 nodes); D/Ca over t >= 3, Ca <= 0.2: 1.04 and 0.84 for the two
    rates, 0.98 jointly (0.95 with the third rate, 3.33e-6); tilt at t = 50
    0.74 and 0.54 rad."""
    from paper_1802_01272_gb300 import eos
    from paper_1802_01272_gb300 import experiments as X
    T, tau, L = 0.8, 1e-2, 6144
    rl, _ = eos.coexistence(T)
    sigma = eos.interface_tension(T, 1e-4)
    runs = {}
    for gdt, ca_paper in ((1.67e-6, 0.18), (5.0e-6, 0.61)):
        gdot = gdt / DT
        ca0 = rl * T * tau * gdot * 26 * DS / sigma
        r = X.sheared_bubble(26, ca0, Lx=L, Ly=L, t_end=50.0, every=0.5, width=0.0,
                             rho_v=0.23967)
        runs[gdt] = r
        print(f"\ngamma_dot dt = {gdt:.3g}: Ca(t = 50) {r.Ca[-1]:.3f} (paper {ca_paper}), "
              f"R {r.R[-1] / DS:.0f} nodes, D {r.D[-1]:.3f}, theta {r.theta[-1]:.3f}")
        assert abs(r.Ca[-1] / ca_paper - 1.0) < 0.15
    C = np.concatenate([r.Ca[(r.t >= 3.0) & (r.Ca <= 0.2)] for r in runs.values()])
    D = np.concatenate([r.D[(r.t >= 3.0) & (r.Ca <= 0.2)] for r in runs.values()])
    slope = float(np.sum(C * D) / np.sum(C * C))
    print(f"D = {slope:.3f} Ca for Ca <= 0.2 (paper's fit 0.89)")
    assert abs(slope - 0.89) < 0.15
    slow, fast = runs[1.67e-6], runs[5.0e-6]
    assert slow.theta[-1] > fast.theta[-1] + 0.1
    areas = [r.R[-1] for r in runs.values()]
    assert max(areas) / min(areas) < 1.15
