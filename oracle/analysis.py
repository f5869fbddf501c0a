"""Closed-form physics of arXiv:1802.01272 used to pin the oracle (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY (tests and benchmark baselines import it).

- free energy psi and vdW pressure ........ Eqs. (free-en2), (evdw)
- Maxwell coexistence densities ........... Sec. II E (equal pressure, equal mu)
- surface tension of the planar interface . Eq. (sigma), read as kappa * int rho'^2 dx
- critical bubble radius .................. Eq. (raggio_c)
- 2D Rayleigh-Plesset ODE (RK4) ........... Eq. (rp)
- CTU1 numerical viscosity ................ Eq. (ctuevol3) projected on a shear wave
- gyration tensor -> a, b, D, theta ....... Eq. (gyr) and Sec. III C
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize


def psi(rho, T, a=9 / 8, b=1 / 3):
    """Bulk free-energy density psi = rho T ln(rho / (1 - b rho)) - a rho^2;
    with b = 1/3 this is Eq. (free-en2), rho T ln(3 rho / (3 - rho)) - 9/8 rho^2."""
    return rho * T * np.log(rho / (1.0 - b * rho)) - a * rho * rho


def mu(rho, T, a=9 / 8, b=1 / 3):
    """d psi / d rho."""
    return T * np.log(rho / (1.0 - b * rho)) + T / (1.0 - b * rho) - 2.0 * a * rho


def p_vdw(rho, T, a=9 / 8, b=1 / 3):
    """Eq. (evdw): p^w = rho dpsi/drho - psi = rho T / (1 - b rho) - a rho^2."""
    return rho * T / (1.0 - b * rho) - a * rho * rho


def dp_drho(rho, T, a=9 / 8, b=1 / 3):
    return T / (1.0 - b * rho) ** 2 - 2.0 * a * rho


def spinodals(T, a=9 / 8, b=1 / 3):
    """Densities where dp/drho = 0 (vapour spinodal < liquid spinodal), T < 1."""
    rc = 1.0  # critical density for a = 9/8, b = 1/3
    lo = optimize.brentq(lambda r: dp_drho(r, T, a, b), 1e-9, rc)
    hi = optimize.brentq(lambda r: dp_drho(r, T, a, b), rc, 1.0 / b - 1e-9)
    return lo, hi


def maxwell(T, a=9 / 8, b=1 / 3):
    """Coexisting (rho_L, rho_V): equal pressure and equal chemical potential."""
    sv, sl = spinodals(T, a, b)
    p_lo = max(p_vdw(sl, T, a, b), 1e-300)   # pressure at the liquid spinodal (local min)
    p_hi = p_vdw(sv, T, a, b)                # pressure at the vapour spinodal (local max)

    def branches(P):
        rv = optimize.brentq(lambda r: p_vdw(r, T, a, b) - P, 1e-300, sv, xtol=1e-16)
        rl = optimize.brentq(lambda r: p_vdw(r, T, a, b) - P, sl, 1.0 / b - 1e-12, xtol=1e-16)
        return rl, rv

    def dmu(P):
        rl, rv = branches(P)
        return mu(rl, T, a, b) - mu(rv, T, a, b)

    eps = 1e-13 * max(1.0, abs(p_hi))
    P = optimize.brentq(dmu, p_lo + eps, p_hi - eps, xtol=1e-16, rtol=1e-15, maxiter=500)
    rl, rv = branches(P)
    return float(rl), float(rv)


def sigma_exact(T, kappa, a=9 / 8, b=1 / 3):
    """Planar-interface tension kappa * int (d rho/dx)^2 dx of the free-energy
    functional Eq. (free-en), evaluated as int sqrt(2 kappa omega(rho)) d rho,
    omega = psi - (common tangent through the coexistence points)."""
    rl, rv = maxwell(T, a, b)
    mc = mu(rl, T, a, b)
    base = psi(rv, T, a, b)

    def om(r):
        return max(0.0, psi(r, T, a, b) - base - mc * (r - rv))

    val, _ = integrate.quad(lambda r: math.sqrt(2.0 * kappa * om(r)), rv, rl, limit=200,
                            epsabs=1e-14, epsrel=1e-12)
    return val


def critical_radius(sigma, rho_ext, T, a=9 / 8, b=1 / 3):
    """Eq. (raggio_c), with the -1 exponent the paper restores:
    R_c = -sigma/2 * { [psi(rho_V) - psi(rho_ext)]
                       + (rho_ext - rho_V)/(rho_L - rho_ext) [psi(rho_L) - psi(rho_ext)] }^-1"""
    rl, rv = maxwell(T, a, b)
    pe = psi(rho_ext, T, a, b)
    br = (psi(rv, T, a, b) - pe) + (rho_ext - rv) / (rl - rho_ext) * (psi(rl, T, a, b) - pe)
    return -sigma / 2.0 / br


def rp_rhs(t, y, r_inf, sigma, rho_l, mu_l, p_b, p_inf):
    """Eq. (rp) solved for d2R/dt2; y = (R, dR/dt); p_b, p_inf callables of t."""
    R, V = y
    lg = math.log(r_inf / R)
    rhs = (p_b(t) - p_inf(t)) / rho_l - sigma / (rho_l * R) - 2.0 * mu_l * V / (rho_l * R)
    rhs += 0.5 * (1.0 - R * R / (r_inf * r_inf)) * V * V
    acc = (rhs / lg - V * V) / R
    return np.array([V, acc])


def rp_integrate(R0, V0, t_end, dt, **kw):
    """Classical fourth-order Runge-Kutta for Eq. (rp). Returns (t, R, dR/dt)."""
    n = int(round(t_end / dt))
    ts = np.linspace(0.0, n * dt, n + 1)
    ys = np.zeros((n + 1, 2))
    ys[0] = (R0, V0)
    for s in range(n):
        t, y = ts[s], ys[s]
        k1 = rp_rhs(t, y, **kw)
        k2 = rp_rhs(t + dt / 2, y + dt / 2 * k1, **kw)
        k3 = rp_rhs(t + dt / 2, y + dt / 2 * k2, **kw)
        k4 = rp_rhs(t + dt, y + dt * k3, **kw)
        ys[s + 1] = y + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return ts, ys[:, 0], ys[:, 1]


def ctu1_numerical_viscosity(xi, w, ds, dt, direction=(1.0, 0.0)):
    """Leading-order CTU1 numerical viscosity of a shear wave with wave vector
    along `direction`: each velocity diffuses with D_a = ds/2 |xi_a| (1 - |xi_a| dt/ds)
    along axis a (Eq. ctuevol3).  With f_k ~ w_k (1 + xi_k.u) the transverse
    momentum picks up sum_k w_k xi_perp^2 (D_x n_x^2 + D_y n_y^2)."""
    n = np.asarray(direction, dtype=np.float64)
    n = n / np.linalg.norm(n)
    perp = np.array([-n[1], n[0]])
    ax, ay = np.abs(xi[:, 0]), np.abs(xi[:, 1])
    Dx = 0.5 * ds * ax * (1.0 - ax * dt / ds)
    Dy = 0.5 * ds * ay * (1.0 - ay * dt / ds)
    xp = xi @ perp
    return float(np.sum(w * xp * xp * (Dx * n[0] ** 2 + Dy * n[1] ** 2)))


def physical_viscosity(rho, T, tau, dt):
    """Eq. (phvisco) nu = rho tau T, with the -dt/2 shift of the explicit
    (forward Euler) collision: T (tau - dt/2) at rho = 1."""
    return rho * T * (tau - dt / 2.0)


def shape_from_sums(nb, sx, sy, sxx, sxy, syy):
    """Eq. (gyr) from bubble-site sums; returns dict(a, b, D, theta, cx, cy).
    a = 2 sqrt(Lambda_M), b = 2 sqrt(Lambda_m), D = (a-b)/(a+b), theta = angle of
    the major eigenvector to the x axis, in (-pi/2, pi/2]."""
    cx, cy = sx / nb, sy / nb
    txx = sxx / nb - cx * cx
    txy = sxy / nb - cx * cy
    tyy = syy / nb - cy * cy
    ev, vec = np.linalg.eigh(np.array([[txx, txy], [txy, tyy]]))
    lm, lM = ev[0], ev[1]
    a, b = 2.0 * math.sqrt(max(lM, 0.0)), 2.0 * math.sqrt(max(lm, 0.0))
    v = vec[:, 1]
    theta = math.atan2(v[1], v[0])
    if theta <= -math.pi / 2:
        theta += math.pi
    elif theta > math.pi / 2:
        theta -= math.pi
    return dict(a=a, b=b, D=(a - b) / (a + b), theta=theta, cx=cx, cy=cy)


def coexistence_from_histogram(counts, lo, hi, rho_values=None, split=1.0, halfwidth=2,
                               peak="bin", smooth_bins=2.0):
    """Coexistence densities from a rho histogram: the peak on each side of
    `split`; if the raw densities are given, each peak is refined to the mean
    of the values within +-halfwidth bins of it (a window 2 halfwidth + 1 bins
    wide).  peak="bin": the highest bin.  peak="smoothed": the vertex of the
    parabola through the three highest values of the histogram smoothed by a
    Gaussian of smooth_bins bins, so that the peak moves continuously with the
    data (the highest raw bin jumps by a whole bin when the top of a broad
    peak is nearly flat, as in a state that is still separating)."""
    counts = np.asarray(counts, dtype=np.float64)
    nb = len(counts)
    edges = np.linspace(lo, hi, nb + 1)
    w = (hi - lo) / nb
    centers = 0.5 * (edges[:-1] + edges[1:])
    if peak == "smoothed":
        r = int(np.ceil(4 * smooth_bins))
        k = np.exp(-0.5 * (np.arange(-r, r + 1) / smooth_bins) ** 2)
        hist = np.convolve(counts, k / k.sum(), mode="same")
    elif peak == "bin":
        hist = counts
    else:
        raise ValueError(peak)
    out = []
    for side in (centers < split, centers >= split):
        idx = np.where(side)[0]
        pk = int(idx[np.argmax(hist[idx])])
        x = float(centers[pk])
        if peak == "smoothed" and 0 < pk < nb - 1:
            y0, y1, y2 = hist[pk - 1], hist[pk], hist[pk + 1]
            den = y0 - 2.0 * y1 + y2
            if den < 0.0:
                x += float(np.clip(0.5 * (y0 - y2) / den, -0.5, 0.5)) * w
        if rho_values is None:
            out.append(x)
        elif peak == "bin":
            l, h = edges[max(pk - halfwidth, 0)], edges[min(pk + halfwidth + 1, nb)]
            sel = rho_values[(rho_values >= l) & (rho_values < h)]
            out.append(float(sel.mean()))
        else:
            l, h = x - (halfwidth + 0.5) * w, x + (halfwidth + 0.5) * w
            sel = rho_values[(rho_values >= l) & (rho_values < h)]
            out.append(float(sel.mean()))
    return out[1], out[0]  # (rho_L, rho_V)
