"""Bubble experiments of Sec. III run on the CUDA path.

* surface tension of a relaxed planar interface, sigma = kappa int (d rho/dx)^2 dx
  (Eq. sigma, in the reading whose values the paper prints), and the
  liquid-vapour phase diagram from such interfaces (Sec. II E);
* the critical radius of Eq. (raggio_c) and the growth or collapse of bubbles
  around it with the density reservoir of Sec. III A, and the lattice's own
  critical radius by bisection on the seed radius as Sec. III A estimates it;
* bubble growth against the two-dimensional Rayleigh-Plesset equation
  (Eq. rp), fed with the pressures measured on the lattice as in Sec. III B;
* a bubble deformed by the shear between moving walls (Sec. III C): shape
  from the gyration tensor (Eq. gyr), deformation D = (a - b)/(a + b), tilt
  angle and capillary number Ca = mu_L gamma_dot R / sigma over time.

Host-side analysis is FP64 numpy; every lattice step, moment and diagnostic
runs in the library.  Lengths are in the paper's units (node spacing ds).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import eos
from .binding import LBM_BC_SHEAR_WALLS, LBM_FP32_SHIFTED, LBM_FP64, Lattice, Params


def free_energy(rho, T, a=9 / 8, b=1 / 3):
    """Bulk free-energy density psi = rho T ln(rho / (1 - b rho)) - a rho^2
    (Eq. free-en2 for b = 1/3, a = 9/8)."""
    return rho * T * np.log(rho / (1.0 - b * rho)) - a * rho * rho


def critical_radius(T, rho_ext, sigma, a=9 / 8, b=1 / 3):
    """Eq. (raggio_c): radius of the bubble that neither grows nor shrinks in
    a liquid held at rho_ext, with the coexistence densities of T."""
    rl, rv = eos.coexistence(T, a, b)
    pe = free_energy(rho_ext, T, a, b)
    brace = (free_energy(rv, T, a, b) - pe) + \
        (rho_ext - rv) / (rl - rho_ext) * (free_energy(rl, T, a, b) - pe)
    return -0.5 * sigma / brace


def rayleigh_plesset(R0, V0, times, p_b, p_inf, r_inf, sigma, rho_l, mu_l, dt=1e-3):
    """Eq. (rp) integrated with the classical fourth-order Runge-Kutta scheme;
    p_b and p_inf are callables of t.  Returns R at `times` (ascending, from 0)."""
    def accel(t, R, V):
        lg = math.log(r_inf / R)
        drive = (p_b(t) - p_inf(t)) / rho_l - sigma / (rho_l * R) - 2.0 * mu_l * V / (rho_l * R)
        return (drive + 0.5 * (1.0 - (R / r_inf) ** 2) * V * V - lg * V * V) / (lg * R)

    out = np.empty(len(times))
    t, R, V = 0.0, float(R0), float(V0)
    for i, te in enumerate(times):
        while t < te - 1e-12:
            h = min(dt, te - t)
            k1r, k1v = V, accel(t, R, V)
            k2r, k2v = V + 0.5 * h * k1v, accel(t + 0.5 * h, R + 0.5 * h * k1r, V + 0.5 * h * k1v)
            k3r, k3v = V + 0.5 * h * k2v, accel(t + 0.5 * h, R + 0.5 * h * k2r, V + 0.5 * h * k2v)
            k4r, k4v = V + h * k3v, accel(t + h, R + h * k3r, V + h * k3v)
            R += h / 6.0 * (k1r + 2 * k2r + 2 * k3r + k4r)
            V += h / 6.0 * (k1v + 2 * k2v + 2 * k3v + k4v)
            t += h
        out[i] = R
    return out


def bubble_fields(Lx, Ly, R, rho_in, rho_out, width=1.0):
    """A circular bubble of radius R nodes centred at (Lx/2, Ly/2): a tanh
    profile of `width` nodes between rho_in (inside) and rho_out (width 0: a
    sharp edge, rho_in for r < R); u = 0."""
    y, x = np.mgrid[0:Ly, 0:Lx].astype(np.float64)
    r = np.hypot(x - Lx / 2.0, y - Ly / 2.0)
    if width > 0:
        rho = 0.5 * (rho_out + rho_in) + 0.5 * (rho_out - rho_in) * np.tanh((r - R) / width)
    else:
        rho = np.where(r < R, rho_in, rho_out)
    return rho, np.zeros_like(rho), np.zeros_like(rho)


def _params(Lx, Ly, T, tau, kappa, ds, precision, rho_ref, **kw):
    return Params(Lx=Lx, Ly=Ly, T=T, tau=tau, kappa=kappa, ds=ds, precision=precision,
                  rho_ref=rho_ref, **kw)


def planar_interface_sigma(T=0.8, kappa=1e-4, ds=1 / 256, Lx=512, Ly=8, tau=1e-3, t_end=50.0,
                           precision=LBM_FP64, stream=None):
    """Eq. (sigma) on a relaxed liquid slab between two vapour regions
    (periodic x): sigma = kappa sum_i (d rho/dx)_i^2 ds per interface, with the
    centred difference of the node densities.  Returns (sigma, rho profile).
    The equilibrium of the forced BGK model drifts with tau (the vapour density
    falls as tau grows), so the default is the paper's tau = 1e-3; the vapour
    side relaxes slowly, hence the long default run."""
    rl, rv = eos.coexistence(T)
    x = np.arange(Lx, dtype=np.float64)
    prof = rv + 0.5 * (rl - rv) * (np.tanh((x - Lx / 4) / 2.0) - np.tanh((x - 3 * Lx / 4) / 2.0))
    rho = np.repeat(prof[None, :], Ly, axis=0)
    p = _params(Lx, Ly, T, tau, kappa, ds, precision, rl)
    with Lattice(p, stream) as L:
        L.init_rho_u(rho, np.zeros_like(rho), np.zeros_like(rho))
        L.step(int(round(t_end / p.dt)))
        r, _, _ = L.moments()
    prof = r.mean(axis=0)
    grad = (np.roll(prof, -1) - np.roll(prof, 1)) / (2.0 * ds)
    return kappa * float(np.sum(grad * grad)) * ds / 2.0, prof


def slab_plateaus(prof):
    """Bulk densities of the slab profile of planar_interface_sigma (liquid on
    [Lx/4, 3Lx/4), vapour outside, periodic): the medians over windows of
    Lx/8 + 1 nodes centred on the liquid's middle (Lx/2) and the vapour's
    (node 0), a quarter of the lattice from either interface, so that the
    over- and undershoots next to a diffuse interface stay out.
    Returns (rho_L, rho_V)."""
    prof = np.asarray(prof, dtype=np.float64)
    n = len(prof)
    hw = n // 16
    idx = np.arange(-hw, hw + 1)
    return float(np.median(prof[(n // 2 + idx) % n])), float(np.median(prof[idx % n]))


def phase_diagram(temperatures, kappa=1e-4, ds=1 / 256, tau=1e-3, Lx=128, t_end=20.0,
                  precision=LBM_FP32_SHIFTED, stream=None):
    """Sec. II E's liquid-vapour phase diagram from relaxed planar interfaces:
    for each T, the liquid and vapour plateau densities of a slab (periodic x,
    `Lx` nodes, relaxed to t_end; slab_plateaus) beside the Maxwell values.
    Returns a list of dicts with T, rho_L, rho_V (plateaus), rho_max, rho_min
    (the profile's extremes), maxwell_L, maxwell_V and sigma."""
    out = []
    for T in temperatures:
        sigma, prof = planar_interface_sigma(T=T, kappa=kappa, ds=ds, Lx=Lx, tau=tau,
                                             t_end=t_end, precision=precision, stream=stream)
        rl, rv = eos.coexistence(T)
        pl, pv = slab_plateaus(prof)
        out.append({"T": float(T), "rho_L": pl, "rho_V": pv, "rho_max": float(prof.max()),
                    "rho_min": float(prof.min()), "maxwell_L": rl, "maxwell_V": rv,
                    "sigma": sigma})
    return out


@dataclass
class BubbleRun:
    t: np.ndarray                 # time
    R: np.ndarray                 # equivalent radius sqrt(N_b / pi) ds
    rho_center: np.ndarray        # rho at the bubble centre
    rho_inf: np.ndarray           # mean rho on the ring r = r_inf
    r_inf: float                  # far-field radius R_BC
    params: Params = field(repr=False, default=None)


def bubble_in_reservoir(R0_nodes, rho_ext, T=0.8, kappa=1e-4, ds=1 / 256, L=1024, tau=1e-3,
                        t_end=4.0, every=0.1, rho_v=None, precision=LBM_FP32_SHIFTED,
                        stream=None, width=1.0) -> BubbleRun:
    """Sec. III A-B: a vapour bubble (rho_v, default the coexistence vapour)
    in a superheated liquid held at rho_ext outside R_BC = [L/2 - 1/(2 ds)] ds
    by the reservoir rescale, seeded as a tanh profile of `width` nodes (a
    step as width -> 0).  Records R(t) from the bubble-site count
    (rho < (rho_V + rho_L)/2), rho at the centre and on the ring r = R_BC."""
    rl, rv = eos.coexistence(T)
    rho_v = rv if rho_v is None else rho_v
    rho, ux, uy = bubble_fields(L, L, R0_nodes, rho_v, rho_ext, width)
    p = _params(L, L, T, tau, kappa, ds, precision, rho_ext, reservoir=1, rho_ext=rho_ext)
    thr = 0.5 * (rl + rv)
    r_inf_nodes = L / 2 - 1.0 / (2.0 * ds)
    n_every = max(1, int(round(every / p.dt)))
    n_rec = int(round(t_end / every))
    t, R, rc, ri = [], [], [], []
    with Lattice(p, stream) as Lt:
        Lt.init_rho_u(rho, ux, uy)
        for i in range(n_rec + 1):
            if i:
                Lt.step(n_every)
            d = Lt.diagnostics(thr, r_inf_nodes)
            t.append(i * n_every * p.dt)
            R.append(math.sqrt(d["nb"] / math.pi) * ds)
            rc.append(d["rho_center"])
            ri.append(d["rho_ring"])
    return BubbleRun(t=np.array(t), R=np.array(R), rho_center=np.array(rc), rho_inf=np.array(ri),
                     r_inf=r_inf_nodes * ds, params=p)


def bubble_fate(run: BubbleRun, t_relax=1.0, margin_nodes=1.0) -> int:
    """+1 if the bubble of a reservoir run grew by more than `margin_nodes`
    after the seed's interface relaxed (t >= t_relax), -1 if it shrank by
    more, 0 if undecided over the run."""
    ds = run.params.ds
    i = int(np.searchsorted(run.t, t_relax - 1e-12))
    change = (run.R[-1] - run.R[min(i, len(run.R) - 1)]) / ds
    return 1 if change > margin_nodes else (-1 if change < -margin_nodes else 0)


def critical_radius_bisection(rho_ext, R_shrink, R_grow, fate=None, **run_kw):
    """Sec. III A's estimate of the lattice's critical radius: the smallest
    seed radius R_g that grows and the largest R_s that shrinks, one node
    apart, give R_c = (R_g + R_s) / 2.  Integer seed radii (nodes) are
    bisected between a bracket R_shrink < R_grow that must shrink and grow;
    `fate(R0)` classifies one seed (default: a bubble_in_reservoir run with
    `run_kw`, judged by bubble_fate; an undecided run raises).  Returns
    (R_s, R_g, R_c, {R0: fate}) in nodes."""
    if fate is None:
        def fate(R0):
            return bubble_fate(bubble_in_reservoir(R0, rho_ext, **run_kw))
    lo, hi = int(R_shrink), int(R_grow)
    if not lo < hi:
        raise ValueError("need R_shrink < R_grow")
    seen = {}
    for r, want in ((lo, -1), (hi, 1)):
        seen[r] = fate(r)
        if seen[r] != want:
            raise ValueError(f"seed {r} does not {'shrink' if want < 0 else 'grow'} "
                             f"(fate {seen[r]}): widen the bracket or the run")
    while hi - lo > 1:
        mid = (lo + hi) // 2
        seen[mid] = fate(mid)
        if seen[mid] == 0:
            raise ValueError(f"seed {mid} undecided: lengthen the run")
        if seen[mid] > 0:
            hi = mid
        else:
            lo = mid
    return lo, hi, 0.5 * (lo + hi), seen


def rp_prediction(run: BubbleRun, t0: float, sigma=None, window=0.5):
    """Sec. III B: integrate Eq. (rp) from the lattice state at t0, after the
    initial interface has relaxed.  R(t0) and dR/dt(t0) come from a straight-line
    fit of the run's R over [t0 - window, t0 + window]; p_B(t) and p_inf(t) are
    the EOS pressures of the measured centre and far-field densities, averaged
    over +-window/2 (the vapour inside rings acoustically); rho_L is the
    coexistence liquid density and mu_L = rho_L T tau.  Returns (t, R_RP) at
    the run's record times >= t0."""
    p = run.params
    rl, _ = eos.coexistence(p.T)
    sigma = eos.interface_tension(p.T, p.kappa) if sigma is None else sigma
    i0 = int(np.searchsorted(run.t, t0 - 1e-12))
    fit = np.abs(run.t - run.t[i0]) <= window + 1e-12
    V0, R0 = np.polyfit(run.t[fit] - run.t[i0], run.R[fit], 1)

    def smooth(x):
        out = np.empty_like(x)
        for j, tj in enumerate(run.t):
            out[j] = x[np.abs(run.t - tj) <= 0.5 * window + 1e-12].mean()
        return out

    pb = eos.pressure(smooth(run.rho_center), p.T)[i0:]
    pf = eos.pressure(smooth(run.rho_inf), p.T)[i0:]
    ts = run.t[i0:] - run.t[i0]
    R = rayleigh_plesset(R0, V0, ts, lambda t: np.interp(t, ts, pb),
                         lambda t: np.interp(t, ts, pf), run.r_inf, sigma, rl, rl * p.T * p.tau)
    return run.t[i0:], R


@dataclass
class ShearRun:
    t: np.ndarray        # time
    D: np.ndarray        # (a - b)/(a + b) from the gyration tensor
    theta: np.ndarray    # tilt of the major axis to the flow direction x
    R: np.ndarray        # mean radius (a + b)/2, lattice units of length
    Ca: np.ndarray       # mu_L gamma_dot R / sigma
    shear_rate: float


def sheared_bubble(R0_nodes, capillary, Lx=1024, Ly=512, T=0.8, kappa=1e-4, ds=1 / 256,
                   tau=1e-2, rho_ext=1.90, t_end=10.0, every=0.5,
                   precision=LBM_FP32_SHIFTED, stream=None, width=2.0,
                   rho_v=None) -> ShearRun:
    """Sec. III C: a vapour bubble (radius R0) growing in a superheated liquid
    (rho_ext, 1.90 as in the paper's runs at T = 0.8, tau = 1e-2) sheared
    between walls moving at -+u_w (y = 0, Ly), periodic in x.  The shear rate
    is set from the target capillary number of the initial radius,
    gamma_dot = Ca sigma / (mu_L R0) with mu_L = rho_L T tau; the fluid starts
    in the linear shear profile.  Records the shape of Eq. (gyr) over time;
    Ca(t) follows the growing mean radius, as in the paper.  The seed is a
    tanh profile of `width` nodes (0: sharp) at rho_v (default: Maxwell's
    vapour density)."""
    rl, rv = eos.coexistence(T)
    sigma = eos.interface_tension(T, kappa)
    mu_l = rl * T * tau
    gdot = capillary * sigma / (mu_l * R0_nodes * ds)
    uw = gdot * Ly * ds / 2.0
    rho, ux, uy = bubble_fields(Lx, Ly, R0_nodes, rv if rho_v is None else rho_v, rho_ext,
                                width)
    y = np.arange(Ly, dtype=np.float64)
    ux = np.repeat((-uw + 2.0 * uw * (y + 1.0) / (Ly + 1.0))[:, None], Lx, axis=1)
    p = _params(Lx, Ly, T, tau, kappa, ds, precision, rho_ext, boundary=LBM_BC_SHEAR_WALLS,
                shear_rate=gdot, rho_ext=rho_ext)
    thr = 0.5 * (rl + rv)
    n_every = max(1, int(round(every / p.dt)))
    t, D, th, R = [], [], [], []
    with Lattice(p, stream) as L:
        L.init_rho_u(rho, ux, uy)
        for i in range(int(round(t_end / every)) + 1):
            if i:
                L.step(n_every)
            d = L.diagnostics(thr)
            t.append(i * n_every * p.dt)
            D.append(d["D"])
            th.append(d["theta"])
            R.append(0.5 * (d["a"] + d["b"]) * ds)
    R = np.array(R)
    return ShearRun(t=np.array(t), D=np.array(D), theta=np.array(th), R=R,
                    Ca=mu_l * gdot * R / sigma, shear_rate=gdot)
