"""Shared test helpers: parameter translation oracle <-> library, error metrics."""
import numpy as np

RHO_L_T09 = 1.657270211998323   # Maxwell liquid density at T = 0.9 (pinned in test_oracle_pins)
RHO_V_T09 = 0.425741637724056


def oracle_params(O, lp):
    """Oracle parameters equal to a library Params."""
    return O.Params(Lx=lp.Lx, Ly=lp.Ly, a=lp.a, b=lp.b, kappa=lp.kappa, T=lp.T, tau=lp.tau,
                    dt=lp.dt, ds=lp.ds, ctu_order=lp.ctu_order, limiter=lp.limiter,
                    regularize=lp.regularize, boundary=lp.boundary, shear_rate=lp.shear_rate,
                    rho_ext=lp.rho_ext, reservoir=lp.reservoir)


def rel_err(a, b):
    """max |a - b| / max |b|  (normwise relative error, safe for fields near 0)."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_err_elem(a, b, floor=1e-3, abs_floor=0.0):
    """max |a - b| / (|b| + floor * max |b| + abs_floor): element-wise relative
    error, with a floor so that entries near zero are compared at a fixed
    scale (a fraction of the field's largest entry, or an absolute scale such
    as the thermal speed sqrt(T) for velocities)."""
    a, b = np.asarray(a), np.asarray(b)
    scale = max(np.abs(b).max(), 1e-300)
    return float((np.abs(a - b) / (np.abs(b) + floor * scale + abs_floor)).max())
