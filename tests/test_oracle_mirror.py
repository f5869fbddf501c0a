"""Pins of the oracle's CTU2 limiter arguments by the x <-> y mirror symmetry of
the method (Sec. II C 2), with mutation checks on altered copies of the oracle.

The printed S^y of Sec. II C 2 carries R^x in the limiter argument; the oracle
reads it as Psi(R^y_{i,j-s_y} / R^y_{i,j}), the mirror image of S^x.  The
16-velocity set of Table I is closed under the exchange of the x and y
components, the lattice is square and periodic, and every other part of the
step (f^eq, F_k, the force stencils) is symmetric under that exchange, so a
step of the transposed state must equal the transposed step.  A misread S^y
breaks this by far more than rounding; the mutation tests below compile the
oracle with each plausible misreading of S^y's argument (the printed R^x, the
downwind neighbour, the x sign of the velocity) and check that the symmetry
test fails for every one of them.

The symmetry ties S^y to S^x; each is also pinned on its own by the reduction
to one dimension: on a single lattice row (or column), without force and
relaxation, CTU2 + MC is the textbook flux-limited high-resolution method for
linear advection (LeVeque 2002, Sec. 6.12), which the test writes in its own
interface form.  (The Table II shear-wave viscosity does not pin the limiter
argument: on a smooth wave the ratio of neighbouring jumps is near 1 either
way, and a downwind argument moves the CTU2 viscosity by only 0.3 %.)
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_SRC = os.path.join(ROOT, "oracle", "ctu_oracle.c")

SY_LINE = "double theta = Ry(L, k, i, j - sgn(XI[k][1])) / r;"
SX_LINE = "double theta = Rx(L, k, i - sgn(XI[k][0]), j) / r;"

# each plausible misreading of the limiter argument, as a one-line substitution
SY_MUTANTS = {
    "printed_Rx": (SY_LINE, "double theta = Rx(L, k, i, j - sgn(XI[k][1])) / Rx(L, k, i, j);"),
    "downwind_row": (SY_LINE, "double theta = Ry(L, k, i, j + sgn(XI[k][1])) / r;"),
    "x_sign": (SY_LINE, "double theta = Ry(L, k, i, j - sgn(XI[k][0])) / r;"),
}


def transpose_velocity_map(xi):
    """perm[k] = index of the velocity (xi_y, xi_x) of velocity k."""
    perm = np.empty(16, dtype=int)
    for k in range(16):
        m = np.where(np.all(np.isclose(xi, xi[k][::-1], rtol=0, atol=1e-14), axis=1))[0]
        assert len(m) == 1
        perm[k] = m[0]
    return perm


def transposed(f, perm):
    g = np.empty_like(f)
    for k in range(16):
        g[perm[k]] = f[k].T
    return g


def rough_state(O, p, seed=11):
    """A noisy liquid near T = 0.9 with every f_k perturbed independently by
    10 %: the jumps R change sign often, so the MC limiter takes all of its
    branches (0, the centred slope, the doubled one-sided slopes)."""
    rho, ux, uy = synth.noisy_uniform(p.Lx, p.Ly, 1.4, 0.05, seed=seed)
    ux = 0.05 * synth.normal(seed + 1, p.Lx * p.Ly).reshape(p.Ly, p.Lx)
    uy = 0.05 * synth.normal(seed + 2, p.Lx * p.Ly).reshape(p.Ly, p.Lx)
    f = O.init_feq(p, rho, ux, uy)
    z = synth.normal(seed + 3, f.size).reshape(f.shape)
    return f * (1.0 + 0.1 * z)


def mirror_error(step, O, p, nsteps=3):
    """max |step(f^T) - step(f)^T| / max |step(f)| over a few steps."""
    xi, _ = O.velocity_set()
    perm = transpose_velocity_map(xi)
    f0 = rough_state(O, p)
    a = step(p, f0, nsteps)
    b = step(p, transposed(f0, perm), nsteps)
    return float(np.abs(b - transposed(a, perm)).max() / np.abs(a).max())


def mutant_step(tmp_path, name, old, new):
    """orc_step of a copy of the oracle with one source line replaced."""
    src = open(ORACLE_SRC).read()
    assert src.count(old) == 1, f"oracle source changed: {old!r} not found once"
    d = tmp_path / name
    d.mkdir()
    (d / "ctu_oracle.c").write_text(src.replace(old, new))
    (d / "ctu_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "ctu_oracle.h")).read())
    so = d / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-o",
                    str(so), str(d / "ctu_oracle.c"), "-lm"], check=True)
    lib = C.CDLL(str(so))
    import oracle as O
    lib.orc_step.argtypes = [C.POINTER(O._Params), C.POINTER(C.c_double), C.c_int64]
    lib.orc_step.restype = C.c_int

    def step(p, f, n):
        f = np.array(f, dtype=np.float64, order="C")
        rc = lib.orc_step(C.byref(p.c()), f.ctypes.data_as(C.POINTER(C.c_double)), int(n))
        assert rc == 0
        return f
    return step


def mirror_params(O):
    return O.Params(Lx=24, Ly=24, T=0.9, tau=1e-3, ctu_order=2, limiter=O.LIM_MC)


def test_ctu2_mc_step_is_mirror_symmetric(oracle_mod):
    """CTU2 + MC with the force: the step commutes with x <-> y to rounding."""
    O = oracle_mod
    err = mirror_error(O.step, O, mirror_params(O))
    assert err < 1e-13, err


def test_mirror_symmetry_holds_for_ctu1_and_fixed_limiters(oracle_mod):
    """The same with CTU1 and with CTU2 at Psi = 1 (the limiter argument unused):
    the symmetry test itself does not depend on the limiter."""
    O = oracle_mod
    for order, lim in ((1, O.LIM_MC), (2, O.LIM_ONE), (2, O.LIM_ZERO)):
        p = mirror_params(O)
        p.ctu_order, p.limiter = order, lim
        assert mirror_error(O.step, O, p) < 1e-13


@pytest.mark.parametrize("name", sorted(SY_MUTANTS))
def test_mirror_symmetry_fails_for_each_misread_Sy(oracle_mod, tmp_path, name):
    """Each misreading of S^y's limiter argument breaks the symmetry by orders
    of magnitude more than rounding: the test above pins reading R1."""
    O = oracle_mod
    old, new = SY_MUTANTS[name]
    step = mutant_step(tmp_path, name, old, new)
    err = mirror_error(step, O, mirror_params(O))
    assert err > 1e-7, (name, err)


def textbook_high_resolution_1d(q, nu):
    """One step of the flux-limited high-resolution method for q_t + u q_x = 0
    with u > 0 on a periodic 1-D grid, in the interface form of LeVeque,
    Finite Volume Methods for Hyperbolic Problems (2002), Sec. 6.12:
        Q_i <- Q_i - nu (Q_i - Q_{i-1})
               - nu (1 - nu)/2 [phi(th_{i+1/2}) dQ_{i+1/2} - phi(th_{i-1/2}) dQ_{i-1/2}],
    dQ_{i-1/2} = Q_i - Q_{i-1}, th_{i-1/2} = dQ_{i-3/2} / dQ_{i-1/2} (the upwind
    interface), phi the MC limiter (phi = 0 where dQ_{i-1/2} = 0)."""
    dq = q - np.roll(q, 1)                       # dQ_{i-1/2}
    up = np.roll(dq, 1)                          # dQ_{i-3/2}
    with np.errstate(divide="ignore", invalid="ignore"):
        th = np.where(dq != 0.0, up / np.where(dq != 0.0, dq, 1.0), 0.0)
    phi = np.maximum(0.0, np.minimum(np.minimum((1.0 + th) / 2.0, 2.0), 2.0 * th))
    phi = np.where(dq != 0.0, phi, 0.0)
    lim = phi * dq                               # limited jump at i-1/2
    return q - nu * dq - 0.5 * nu * (1.0 - nu) * (np.roll(lim, -1) - lim)


def advect_1d_reference(O, p, f, axis):
    """Each f_k advected one step by the textbook method along `axis`
    (1: x, 0: y of the [Ly][Lx] plane), the velocity's sign by reversal."""
    xi, _ = O.velocity_set()
    out = np.empty_like(f)
    d = 0 if axis == 1 else 1
    for k in range(16):
        c = abs(xi[k][d]) * p.dt / p.ds
        q = f[k].reshape(-1)
        if xi[k][d] > 0:
            out[k] = textbook_high_resolution_1d(q, c).reshape(f[k].shape)
        else:
            out[k] = textbook_high_resolution_1d(q[::-1], c)[::-1].reshape(f[k].shape)
    return out


def one_d_case(O, axis, seed=5):
    """A rough 1-D state (every f_k independent noise) with no force (a = b =
    kappa = 0, so p^i - p^w = 0) and no relaxation (tau = 1e30: dt/tau = 1e-34)."""
    n = 48
    Lx, Ly = (n, 1) if axis == 1 else (1, n)
    p = O.Params(Lx=Lx, Ly=Ly, a=0.0, b=0.0, kappa=0.0, T=1.0, tau=1e30, ctu_order=2,
                 limiter=O.LIM_MC)
    z = synth.normal(seed, 16 * n).reshape(16, Ly, Lx)
    f = 0.05 + 0.02 * z
    # a few plateaus and a jump, so that th = 0, negative th and dQ = 0 all occur
    f[:, :, :] = np.where(np.abs(z) < 0.3, 0.05, f)
    return p, f


@pytest.mark.parametrize("axis", [1, 0], ids=["x", "y"])
def test_ctu2_reduces_to_textbook_high_resolution_method_in_1d(oracle_mod, axis):
    """With one lattice row (or column), no force and no relaxation, a CTU2 + MC
    step is the 1-D flux-limited method for linear advection applied to each
    f_k with Courant number |xi| dt / ds: S^x (S^y) with its upwind limiter
    argument, and nothing from the transverse terms."""
    O = oracle_mod
    p, f = one_d_case(O, axis)
    got = O.step(p, f, 1)
    ref = advect_1d_reference(O, p, f, axis)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-13


LIMITER_MUTANTS = {
    "x_downwind": (1, SX_LINE, "double theta = Rx(L, k, i + sgn(XI[k][0]), j) / r;"),
    "x_y_sign": (1, SX_LINE, "double theta = Rx(L, k, i - sgn(XI[k][1]), j) / r;"),
    "y_printed_Rx": (0,) + SY_MUTANTS["printed_Rx"],
    "y_downwind": (0,) + SY_MUTANTS["downwind_row"],
    "y_x_sign": (0,) + SY_MUTANTS["x_sign"],
}


@pytest.mark.parametrize("name", sorted(LIMITER_MUTANTS))
def test_1d_reduction_fails_for_each_misread_limiter_argument(oracle_mod, tmp_path, name):
    """The 1-D reduction rejects every misreading of the limiter arguments."""
    O = oracle_mod
    axis, old, new = LIMITER_MUTANTS[name]
    step = mutant_step(tmp_path, name, old, new)
    p, f = one_d_case(O, axis)
    got = step(p, f, 1)
    ref = advect_1d_reference(O, p, f, axis)
    assert np.abs(got - ref).max() / np.abs(ref).max() > 1e-6, name
