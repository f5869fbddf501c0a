"""Parity at the benchmark's full size and launch configuration.

The 6144 x 6144 sheared-bubble workload of bench.py (FP32 shifted storage,
CTU2 + MC, shear walls) is stepped on the GPU.  One step of a node depends on
f^n within 4 nodes (advection radius 2, then the 5x5 force stencil on the
advected density), so a window of the GPU's f^n with a halo of 4 nodes per
step, stepped by the oracle, reproduces the GPU's interior exactly up to
rounding.  Windows sit on both walls, across the periodic x seam, across
strip seams of the kernel's decomposition and on the bubble interface.
"""
import numpy as np
import pytest

from tests.conftest import has_gpu
from tests.helpers import rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]

HALO = 4  # dependency radius of one step


def _window(full, y0, x0, h, w):
    import torch
    Ly, Lx = full.shape[1], full.shape[2]
    iy = torch.arange(y0, y0 + h, device=full.device) % Ly
    ix = torch.arange(x0, x0 + w, device=full.device) % Lx
    return full.index_select(1, iy).index_select(2, ix).cpu().numpy()


def _check_windows(P, O, lp, windows, nsteps, tol):
    import torch
    import bench
    w = bench.WORKLOADS["sheared-bubble-6144"]
    rho, ux, uy = bench.initial_fields(w, lp.Lx, lp.Ly)
    stream = torch.cuda.current_stream()
    with P.Lattice(lp, stream) as L:
        L.init_rho_u(rho, ux, uy)
        L.step(3)                      # a state with developed non-equilibrium parts
        f0 = torch.empty((16, lp.Ly, lp.Lx), dtype=torch.float64, device="cuda")
        L.get_f_device(f0)
        L.step(nsteps)
        f1 = torch.empty_like(f0)
        L.get_f_device(f1)
        L.sync()
    halo = HALO * nsteps
    uw = lp.shear_rate * lp.Ly * lp.ds / 2.0
    worst = 0.0
    for (y0, x0, h, wd, wall_bottom, wall_top) in windows:
        ya = y0 if wall_bottom else y0 - halo
        yb = y0 + h if wall_top else y0 + h + halo
        win = _window(f0, ya, x0 - halo, yb - ya, wd + 2 * halo)
        Hy, Wx = win.shape[1], win.shape[2]
        walls = wall_bottom or wall_top
        op = O.Params(Lx=Wx, Ly=Hy, a=lp.a, b=lp.b, kappa=lp.kappa, T=lp.T, tau=lp.tau, dt=lp.dt,
                      ds=lp.ds, ctu_order=lp.ctu_order, limiter=lp.limiter,
                      boundary=O.BC_SHEAR_WALLS if walls else O.BC_PERIODIC,
                      shear_rate=2 * uw / (Hy * lp.ds) if walls else 0.0, rho_ext=lp.rho_ext)
        out = O.step(op, win, nsteps)
        oy = y0 - ya
        got = _window(f1, y0, x0, h, wd)
        ref = out[:, oy:oy + h, halo:halo + wd]
        e = rel_err(got, ref)
        worst = max(worst, e)
        assert e < tol, f"window y0={y0} x0={x0}: {e:.2e}"
    return worst


def _params(P, precision):
    import bench
    w = bench.WORKLOADS["sheared-bubble-6144"]
    lp = bench.lib_params(P, w)
    lp.precision = precision
    return lp


WINDOWS = [
    # (y0, x0, height, width, touches bottom wall, touches top wall)
    (0, 100, 12, 24, True, False),          # bottom wall
    (6144 - 12, 3000, 12, 24, False, True),  # top wall
    (2000, 6144 - 10, 16, 24, False, False),  # periodic x seam
    (4000, 56 * 55 - 8, 16, 24, False, False),  # strip seam of the kernel (56-column strips)
    (3072 - 30, 3072 - 12, 24, 24, False, False),  # bubble interface (R = 26 nodes)
    (1234, 777, 16, 20, False, False),
]


def test_fullsize_fp32_bench_config_windows(oracle_mod):
    import paper_1802_01272_gb300 as P
    lp = _params(P, P.LBM_FP32_SHIFTED)
    worst = _check_windows(P, oracle_mod, lp, WINDOWS, nsteps=10, tol=1e-5)
    print(f"\nFP32 windows after 10 steps: worst {worst:.2e}")
    assert worst < 1e-5


def test_fullsize_fp64_windows(oracle_mod):
    import paper_1802_01272_gb300 as P
    lp = _params(P, P.LBM_FP64)
    worst = _check_windows(P, oracle_mod, lp, WINDOWS[:4], nsteps=4, tol=1e-11)
    assert worst < 1e-11


def test_fullsize_mass_conservation_periodic():
    """Any size: with periodic boundaries the total mass is conserved; FP32
    storage keeps it to ~1e-7 relative per step."""
    import torch
    import bench
    import paper_1802_01272_gb300 as P
    w = dict(bench.WORKLOADS["sheared-bubble-6144"])
    w["walls"] = False
    lp = bench.lib_params(P, w)
    rho, ux, uy = bench.initial_fields(w, lp.Lx, lp.Ly)
    with P.Lattice(lp, torch.cuda.current_stream()) as L:
        L.init_rho_u(rho, ux, uy)
        m0 = L.diagnostics(threshold=1.0)["mass"]
        L.step(10)
        d = L.diagnostics(threshold=1.0)
    assert abs(d["mass"] - m0) / m0 < 1e-6
    assert d["rho_min"] > 0.2 and d["rho_max"] < 2.0
