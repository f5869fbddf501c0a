"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 storage: max relative error <= 1e-11 on f, rho and u (rounding order and
FMA contraction are the only differences).  FP32 shifted storage: <= 1e-5
relative on rho after 1000 steps.
"""
import numpy as np
import pytest

import synth
from tests.conftest import has_gpu
from tests.helpers import RHO_L_T09, oracle_params, rel_err, rel_err_elem

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]

TOL64 = 1e-11


@pytest.fixture(scope="module")
def P():
    import paper_1802_01272_gb300 as P
    P.lib()
    return P


def run_both(P, O, lp, f0, nsteps_list):
    """Advance library and oracle from the same f0; yield (n, f_gpu, f_oracle)."""
    op = oracle_params(O, lp)
    with P.Lattice(lp) as L:
        L.set_f(f0)
        fo = f0.copy()
        done = 0
        for n in nsteps_list:
            L.step(n - done)
            fo = O.step(op, fo, n - done)
            done = n
            yield n, L.get_f(), fo, L


def test_config1_fp64_128_200_steps(P, oracle_mod):
    """128x128, FP64, CTU2 + MC, T = 0.9, rho = rho_L (1 + 1e-3 N(0,1)) seed 0, f = f^eq."""
    O = oracle_mod
    lp = P.Params(Lx=128, Ly=128, precision=P.LBM_FP64, T=0.9)
    rho, ux, uy = synth.noisy_uniform(128, 128, RHO_L_T09, 1e-3, seed=0)
    op = oracle_params(O, lp)
    f0 = O.init_feq(op, rho, ux, uy)
    with P.Lattice(lp) as L:
        L.init_rho_u(rho, ux, uy)
        assert rel_err(L.get_f(), f0) < 1e-14
        fo = f0
        for n in (100, 100):
            L.step(n)
            fo = O.step(op, fo, n)
            fg = L.get_f()
            assert rel_err(fg, fo) < TOL64
            rg, uxg, uyg = L.moments()
            ro, uxo, uyo = O.moments(op, fo)
            assert rel_err(rg, ro) < TOL64
            assert rel_err(uxg, uxo) < TOL64 and rel_err(uyg, uyo) < TOL64
            # element by element: rho relative, u relative to |u| + sqrt(T) (the
            # thermal speed: rounding of f moves u by ~1e-16 of it wherever u ~ 0)
            ct = np.sqrt(lp.T)
            assert rel_err_elem(rg, ro) < TOL64
            assert rel_err_elem(uxg, uxo, 0.0, ct) < TOL64 and rel_err_elem(uyg, uyo, 0.0, ct) < TOL64
        d = L.diagnostics(threshold=1.0)
        assert abs(d["mass"] - ro.sum()) / ro.sum() < 1e-12


CASES = [
    # (Lx, Ly, order, limiter, boundary, reservoir, regularize)
    (100, 70, 2, 0, 0, 0, 0),      # several strips, ragged tail in x and y
    (100, 70, 1, 0, 0, 0, 0),
    (64, 48, 2, 1, 0, 0, 0),       # Psi = 0
    (64, 48, 2, 2, 0, 0, 0),       # Psi = 1
    (37, 23, 2, 0, 0, 0, 0),       # Lx % 4 != 0: scalar path
    (8, 8, 2, 0, 0, 0, 0),         # one strip wider than the lattice
    (64, 3, 2, 0, 0, 0, 0),        # fewer rows than the stencil
    (124, 40, 2, 0, 1, 0, 0),      # shear walls
    (124, 40, 1, 0, 1, 0, 0),
    (300, 300, 2, 0, 0, 1, 0),     # reservoir (R_BC = 22 nodes at ds = 1/256)
    (60, 44, 2, 0, 0, 0, 1),       # regularisation
    (60, 44, 2, 0, 1, 0, 1),
    # interior strips staged by tensor copies; Ly not a multiple of the 4-row
    # batches, several row blocks (96 rows each) of a work item
    (240, 150, 2, 0, 0, 0, 0),
    (240, 200, 2, 0, 1, 0, 0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_variants_fp64(P, oracle_mod, case):
    O = oracle_mod
    Lx, Ly, order, lim, bc, res, reg = case
    lp = P.Params(Lx=Lx, Ly=Ly, precision=P.LBM_FP64, ctu_order=order, limiter=lim, boundary=bc,
                  reservoir=res, regularize=reg, T=0.85, tau=2e-3, rho_ext=1.55)
    if bc:
        lp.shear_rate = 2 * 0.3 / (Ly * lp.ds)     # u_w = 0.3
    rho, ux, uy = synth.bubble(Lx, Ly, 1.55, 0.55, R=min(Lx, Ly) / 4, W=2.0)
    ux = ux + 0.05 * synth.fourier_mode(Lx, Ly, 0.0, 1.0, 1, 2)
    uy = uy - 0.04 * synth.fourier_mode(Lx, Ly, 0.0, 1.0, 2, 1)
    op = oracle_params(O, lp)
    f0 = O.init_feq(op, rho, ux, uy)
    for n, fg, fo, L in run_both(P, O, lp, f0, [1, 7, 40]):
        assert rel_err(fg, fo) < TOL64, f"after {n} steps"
        rg, uxg, uyg = L.moments()
        ro, uxo, uyo = O.moments(oracle_params(O, lp), fo)
        ct = np.sqrt(lp.T)
        assert rel_err_elem(rg, ro) < TOL64, f"rho after {n} steps"
        assert (rel_err_elem(uxg, uxo, 0.0, ct) < TOL64 and
                rel_err_elem(uyg, uyo, 0.0, ct) < TOL64), f"u after {n} steps"


def test_kernel_info_staging_paths(P):
    """Lattices with Lx a multiple of 4 and at least 72 wide stage their
    interior strips with tensor copies; others use per-thread copies only."""
    for (Lx, Ly, prec, want) in ((240, 200, P.LBM_FP64, 1), (240, 200, P.LBM_FP32_SHIFTED, 1),
                                 (6144, 64, P.LBM_FP32_SHIFTED, 1), (37, 23, P.LBM_FP64, 0),
                                 (64, 48, P.LBM_FP32_SHIFTED, 0)):
        with P.Lattice(P.Params(Lx=Lx, Ly=Ly, precision=prec)) as L:
            k = L.kernel_info()
        assert k["tensor_copies"] == want, (Lx, Ly, prec, k)
        assert k["threads"] == 256 and k["strips"] == (Lx + 55) // 56 and k["grid"] >= 1
        assert 16 <= k["row_block"] <= 256


def test_fp32_shifted_1000_steps(P, oracle_mod):
    O = oracle_mod
    lp = P.Params(Lx=96, Ly=80, precision=P.LBM_FP32_SHIFTED, rho_ref=RHO_L_T09, T=0.9)
    rho, ux, uy = synth.noisy_uniform(lp.Lx, lp.Ly, RHO_L_T09, 1e-2, seed=5)
    op = oracle_params(O, lp)
    f0 = O.init_feq(op, rho, ux, uy)
    with P.Lattice(lp) as L:
        L.init_rho_u(rho, ux, uy)
        L.step(1000)
        rg, _, _ = L.moments()
    ro, _, _ = O.moments(op, O.step(op, f0, 1000))
    assert rel_err(rg, ro) < 1e-5


def test_fp32_bubble_with_walls(P, oracle_mod):
    """FP32 shifted storage against the FP64 oracle on a bubble between moving
    walls (tau = 1e-2, u_w = 0.2): rho within 1e-5 normwise after 1000 and
    2000 steps.  Element by element the vapour nodes carry more: the stored
    deviations f - w rho_ref are rounded relative to rho_ref = 1.9, which is
    8 times the vapour's 0.24, and u = j / rho carries the same factor.  So
    element-wise rho (relative to |rho|) and u (relative to |u| + sqrt(T))
    are held to 2e-5 after 1000 steps and 4e-5 after 2000 (measured 1.1e-5,
    1.3e-5 and 1.3e-5, 1.6e-5: the rounding accumulates about linearly)."""
    O = oracle_mod
    lp = P.Params(Lx=128, Ly=96, precision=P.LBM_FP32_SHIFTED, rho_ref=1.9, T=0.8, tau=1e-2,
                  boundary=P.LBM_BC_SHEAR_WALLS, rho_ext=1.9)
    lp.shear_rate = 2 * 0.2 / (lp.Ly * lp.ds)
    rho, ux, uy = synth.bubble(lp.Lx, lp.Ly, 1.9, 0.24, R=20, W=4)
    ux = synth.linear_shear(lp.Lx, lp.Ly, 0.2)
    op = oracle_params(O, lp)
    fo = O.init_feq(op, rho, ux, uy)
    ct = np.sqrt(lp.T)
    with P.Lattice(lp) as L:
        L.init_rho_u(rho, ux, uy)
        for n, bar in ((1000, 2e-5), (2000, 4e-5)):
            L.step(1000)
            fo = O.step(op, fo, 1000)
            rg, uxg, uyg = L.moments()
            ro, uxo, uyo = O.moments(op, fo)
            e_rho = rel_err_elem(rg, ro)
            e_u = max(rel_err_elem(uxg, uxo, 0.0, ct), rel_err_elem(uyg, uyo, 0.0, ct))
            print(f"\nFP32 vs oracle after {n} steps: rho {rel_err(rg, ro):.2e} (element-wise "
                  f"{e_rho:.2e}), u {e_u:.2e} relative to |u| + sqrt(T)")
            assert rel_err(rg, ro) < 1e-5 and e_rho < bar and e_u < bar, n


def test_checkpoint_resume_bit_identical(P):
    for prec in (P.LBM_FP64, P.LBM_FP32_SHIFTED):
        lp = P.Params(Lx=64, Ly=40, precision=prec)
        rho, ux, uy = synth.noisy_uniform(64, 40, 1.2, 0.02, seed=2)
        with P.Lattice(lp) as A, P.Lattice(lp) as B:
            A.init_rho_u(rho, ux, uy)
            B.init_rho_u(rho, ux, uy)
            A.step(30)
            B.step(12)
            ck = B.get_f()
            B.set_f(ck)
            B.step(18)
            assert np.array_equal(A.get_f(), B.get_f())


def test_diagnostics_match_oracle(P, oracle_mod):
    O = oracle_mod
    lp = P.Params(Lx=160, Ly=140, precision=P.LBM_FP64, T=0.8)
    rho, ux, uy = synth.bubble(160, 140, 1.9, 0.24, R=30, W=3, cx=81.3, cy=66.7)
    op = oracle_params(O, lp)
    f = O.init_feq(op, rho, ux, uy)
    with P.Lattice(lp) as L:
        L.set_f(f)
        d = L.diagnostics(threshold=(1.9 + 0.24) / 2, r_ring=50.0)
        h = L.histogram(256, 0.0, 3.0)
    o = O.diagnostics(op, f, (1.9 + 0.24) / 2, 50.0)
    assert abs(d["mass"] - o["mass"]) / o["mass"] < 1e-12   # 22400-term sums, two orders
    for n in ("nb", "sx", "sy", "sxx", "sxy", "syy"):
        assert d[n] == int(o[n])
    for n in ("rho_center", "rho_ring", "rho_min", "rho_max"):
        assert abs(d[n] - o[n]) < 1e-13
    assert np.array_equal(h, O.histogram(op, f, 256, 0.0, 3.0))
    from oracle import analysis as A
    s = A.shape_from_sums(o["nb"], o["sx"], o["sy"], o["sxx"], o["sxy"], o["syy"])
    for n in ("a", "b", "D"):
        assert abs(d[n] - s[n]) < 1e-9
    assert abs(np.tan(d["theta"] - s["theta"])) < 1e-6


def test_nonfinite_state_is_reported(P):
    lp = P.Params(Lx=32, Ly=32, precision=P.LBM_FP64)
    rho, ux, uy = synth.noisy_uniform(32, 32, 1.0, 0.0, seed=0)
    with P.Lattice(lp) as L:
        L.init_rho_u(rho, ux, uy)
        f = L.get_f()
        f[:, 5, 7] = np.nan
        L.set_f(f)
        L.step(1)
        with pytest.raises(P.LBMError) as e:
            L.sync()
        assert e.value.code == -7
        L.sync()  # the sticky error was cleared


def test_zero_steps_and_step_count(P):
    lp = P.Params(Lx=16, Ly=16)
    rho, ux, uy = synth.noisy_uniform(16, 16, 1.0, 0.01, seed=1)
    with P.Lattice(lp) as L:
        L.init_rho_u(rho, ux, uy)
        f0 = L.get_f()
        L.step(0)
        assert np.array_equal(L.get_f(), f0) and L.step_count == 0
        L.step(3)
        assert L.step_count == 3


def test_step_many_matches_stepping_alone(P):
    """Lattices of different sizes and physics stepped by one batched launch per
    step end where they end when stepped alone, to FP32 rounding (the batched
    and single kernels are compiled separately, so the compiler may fuse
    multiply-adds differently); an FP64 lattice in the list steps on its own and
    is bitwise equal."""
    import torch
    from paper_1802_01272_gb300.binding import step_many
    stream = torch.cuda.current_stream()
    specs = [
        dict(Lx=256, Ly=200, T=0.9, tau=1e-3),
        dict(Lx=512, Ly=96, T=0.8, tau=1e-2, boundary=P.LBM_BC_SHEAR_WALLS, rho_ext=1.9,
             shear_rate=2 * 0.2 / (96 / 256.0)),
        dict(Lx=128, Ly=300, T=0.95, tau=2e-3),
        dict(Lx=64, Ly=64, T=0.9, precision=P.LBM_FP64),
    ]
    def make(spec, seed):
        lp = P.Params(rho_ref=1.2, **spec)
        L = P.Lattice(lp, stream)
        rho, ux, uy = synth.bubble(lp.Lx, lp.Ly, 1.5, 0.6, R=min(lp.Lx, lp.Ly) / 5, W=2)
        L.init_rho_u(rho * (1 + 1e-3 * synth.normal(seed, lp.Lx * lp.Ly).reshape(rho.shape)),
                     ux, uy)
        return L
    alone = [make(s, i) for i, s in enumerate(specs)]
    mixed = [make(s, i) for i, s in enumerate(specs)]
    for L in alone:
        L.step(9)
    step_many(mixed, 4)
    step_many(mixed, 5)
    for A, B in zip(alone, mixed):
        assert A.step_count == B.step_count == 9
        fa, fb = A.get_f(), B.get_f()
        if A.params.precision == P.LBM_FP64:
            assert np.array_equal(fa, fb)
        else:
            err = rel_err(fb, fa)
            print(f"batched vs alone {A.params.Lx}x{A.params.Ly}: {err:.2e}")
            assert err < 1e-5
    for L in alone + mixed:
        L.close()


def test_step_diag_fused_record_matches_full_diagnostics(P):
    """Diagnostics reduced inside the last step equal the separate reduction of
    the state after it (FP64: same sites, same integer sums, mass to rounding)."""
    for prec, tol in ((P.LBM_FP64, 1e-12), (P.LBM_FP32_SHIFTED, 1e-6)):
        lp = P.Params(Lx=300, Ly=260, precision=prec, T=0.8, rho_ref=1.9, rho_ext=1.9,
                      boundary=P.LBM_BC_SHEAR_WALLS, shear_rate=2 * 0.1 / (260 / 256.0))
        rho, ux, uy = synth.bubble(300, 260, 1.9, 0.24, R=40, W=3)
        thr = 0.5 * (1.9 + 0.24)
        with P.Lattice(lp) as L:
            L.init_rho_u(rho, ux, uy)
            d = L.step_diag(6, thr)
            full = L.diagnostics(thr)
            assert L.step_count == 6
        assert abs(d["mass"] - full["mass"]) / full["mass"] < tol
        if prec == P.LBM_FP64:
            for n in ("nb", "sx", "sy", "sxx", "sxy", "syy"):
                assert d[n] == full[n]
        else:
            assert abs(d["nb"] - full["nb"]) <= 2
        for n in ("a", "b", "D"):
            assert abs(d[n] - full[n]) < 1e-2 * max(1.0, abs(full[n]))
        assert np.isnan(d["rho_min"]) and not np.isnan(full["rho_min"])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_launched_steps_equal_single_launches(P, prec):
    """lbm_step(n >= 32) sends blocks of 16 steps as one CUDA graph launch: the
    same kernels in the same order, so the state is bit-identical to stepping
    one launch at a time (from either buffer parity)."""
    precision = P.LBM_FP64 if prec == "fp64" else P.LBM_FP32_SHIFTED
    lp = P.Params(Lx=200, Ly=120, precision=precision, T=0.85, rho_ref=1.6, rho_ext=1.6,
                  boundary=P.LBM_BC_SHEAR_WALLS, shear_rate=2 * 0.1 / (120 / 256.0))
    rho, ux, uy = synth.bubble(200, 120, 1.6, 0.5, R=25, W=2)
    with P.Lattice(lp) as A, P.Lattice(lp) as B:
        A.init_rho_u(rho, ux, uy)
        B.init_rho_u(rho, ux, uy)
        A.step(1)
        A.step(50)           # odd start parity, 3 graph launches + 2 single steps
        A.step(40)           # even start parity
        for _ in range(91):
            B.step(1)
        assert A.step_count == B.step_count == 91
        assert np.array_equal(A.get_f(), B.get_f())


def test_tune_picks_a_geometry_and_keeps_results(P):
    """lbm_tune times launch geometries with real steps; the state after the
    same number of steps is bit-identical to an untuned run (the arithmetic
    of a node does not depend on how rows are split into work items)."""
    for precision in (P.LBM_FP64, P.LBM_FP32_SHIFTED):
        lp = P.Params(Lx=300, Ly=260, precision=precision, T=0.85, rho_ref=1.6)
        rho, ux, uy = synth.noisy_uniform(300, 260, 1.6, 1e-2, seed=7)
        with P.Lattice(lp) as A, P.Lattice(lp) as B:
            A.init_rho_u(rho, ux, uy)
            B.init_rho_u(rho, ux, uy)
            k = A.tune(2)
            n = A.step_count
            assert n >= 2 * 4
            assert k == A.kernel_info() and 16 <= k["row_block"] <= 1024
            A.step(40)
            B.set_launch(24, 1)          # any geometry: the same state
            B.step(n + 40)
            assert B.kernel_info()["row_block"] == 24
            assert np.array_equal(A.get_f(), B.get_f())
