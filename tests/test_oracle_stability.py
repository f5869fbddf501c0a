"""The linear stability limit of the method in uniform flow, on the oracle:
the 16-velocity third-order model advanced with CTU2 + MC (T = 0.8,
tau = 1e-2, dt = 1e-4, ds = 1/256) damps a small density perturbation of a
liquid moving at u = 0.8 and amplifies it at u = 0.85 (u / sqrt(T) ~ 0.95;
the perturbation grows about fivefold per 1000 steps).  This bounds the wall
speeds of the sheared-bubble runs; the paper's (Sec. III C: u_w <= 0.6, Mach
~0.5 in the liquid) lie below it."""
import numpy as np
import pytest

import oracle as O


def perturbation_growth(u, L=16):
    """Growth of the density perturbation's standard deviation from step 2000
    to step 4000 (after the damped modes of the seeded noise have decayed)."""
    p = O.Params(Lx=L, Ly=L, T=0.8, tau=1e-2)
    rng = np.random.default_rng(1)
    rho = 1.90 * (1.0 + 1e-6 * rng.standard_normal((L, L)))
    f = O.init_feq(p, rho, np.full((L, L), u), np.zeros((L, L)))
    f = O.step(p, f, 2000)
    r0 = np.std(O.moments(p, f)[0])
    f = O.step(p, f, 2000)
    return float(np.std(O.moments(p, f)[0]) / r0)


@pytest.mark.parametrize("u, grows", [(0.8, False), (0.85, True)])
def test_uniform_flow_stability_limit(u, grows):
    g = perturbation_growth(u)
    print(f"\nu = {u}: perturbation x{g:.3g} from step 2000 to 4000")
    assert (g > 10.0) if grows else (g < 0.5)
