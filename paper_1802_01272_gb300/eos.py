"""Van der Waals equation of state helpers for setting up runs.

p^w = rho T / (1 - b rho) - a rho^2 (Eq. evdw; a = 9/8, b = 1/3 put the
critical point at rho_c = T_c = 1).  Coexistence densities follow the Maxwell
equal-area rule on the (1/rho, p) isotherm; the planar-interface tension of
the square-gradient free energy (Eq. free-en) is kappa * int (d rho / dx)^2 dx.
Host-side utilities (FP64, scipy); the step itself runs in the CUDA library.
"""
from __future__ import annotations

import math

from scipy import integrate, optimize


def pressure(rho, T, a=9 / 8, b=1 / 3):
    return rho * T / (1.0 - b * rho) - a * rho * rho


def _dpdrho(rho, T, a, b):
    return T / (1.0 - b * rho) ** 2 - 2.0 * a * rho


def spinodal_densities(T, a=9 / 8, b=1 / 3):
    """(vapour, liquid) spinodal densities, where dp/drho = 0 (T < T_c)."""
    rc = 1.0 / (3.0 * b)
    v = optimize.brentq(lambda r: _dpdrho(r, T, a, b), 1e-12, rc)
    l = optimize.brentq(lambda r: _dpdrho(r, T, a, b), rc, 1.0 / b - 1e-12)
    return v, l


def coexistence(T, a=9 / 8, b=1 / 3):
    """(rho_L, rho_V) from the equal-area rule: for the coexistence pressure P,
    int_{v_L}^{v_V} (p(v) - P) dv = 0 over specific volume v = 1/rho."""
    sv, sl = spinodal_densities(T, a, b)

    def roots(P):
        rv = optimize.brentq(lambda r: pressure(r, T, a, b) - P, 1e-300, sv, xtol=1e-15)
        rl = optimize.brentq(lambda r: pressure(r, T, a, b) - P, sl, 1.0 / b - 1e-13, xtol=1e-15)
        return rl, rv

    def area(P):
        rl, rv = roots(P)
        vl, vv = 1.0 / rl, 1.0 / rv
        # int p dv in closed form: p(v) = T/(v - b) - a/v^2
        ip = T * math.log((vv - b) / (vl - b)) + a * (1.0 / vv - 1.0 / vl)
        return ip - P * (vv - vl)

    lo = max(pressure(sl, T, a, b), 1e-300)
    hi = pressure(sv, T, a, b)
    eps = 1e-12 * max(abs(hi), 1.0)
    P = optimize.brentq(area, lo + eps, hi - eps, xtol=1e-16, rtol=1e-15, maxiter=500)
    return roots(P)


def interface_tension(T, kappa, a=9 / 8, b=1 / 3):
    """kappa * int rho'^2 dx of the relaxed planar interface, written as
    int_{rho_V}^{rho_L} sqrt(2 kappa Delta(rho)) d rho with Delta the height
    of the bulk free energy above its common tangent."""
    rl, rv = coexistence(T, a, b)

    def f(r):  # bulk free energy density rho T ln(rho/(1 - b rho)) - a rho^2
        return r * T * math.log(r / (1.0 - b * r)) - a * r * r

    slope = (f(rl) - f(rv)) / (rl - rv)
    val, _ = integrate.quad(lambda r: math.sqrt(max(2.0 * kappa * (f(r) - f(rv) - slope * (r - rv)), 0.0)),
                            rv, rl, limit=200, epsabs=1e-14, epsrel=1e-12)
    return val
