"""The continuous-batching sweep server: jobs admitted by memory footprint,
advanced together, each result the one it has alone (to FP32 rounding)."""
import numpy as np
import pytest

import synth
from tests.conftest import has_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]


def make_jobs(P, S, n=7, seed=4):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        L = int(rng.choice([64, 128, 192, 256]))
        T = float(rng.uniform(0.8, 0.95))
        lp = P.Params(Lx=L, Ly=L, T=T, tau=1e-3, rho_ext=1.6, rho_ref=1.6)
        rho, ux, uy = synth.bubble(L, L, 1.6, 0.5, R=L / 6, W=2)
        jobs.append(S.Job(params=lp, rho=rho, ux=ux, uy=uy, nsteps=int(rng.integers(100, 400)),
                          arrival=0.002 * i, diag_threshold=1.0, keep_rho=True))
    return jobs


def test_server_results_equal_alone_and_admission_respects_budget():
    import torch
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import server as S
    stream = torch.cuda.current_stream()
    jobs = make_jobs(P, S)
    budget = 3 * max(j.footprint() for j in jobs)        # at most ~3 resident at once
    srv = S.SweepServer(budget, stream=stream, chunk=64)
    peak = []
    orig_admit = srv._admit

    def admit(now):
        orig_admit(now)
        peak.append(srv.used)
        assert srv.used <= budget
    srv._admit = admit
    for j in jobs:
        srv.submit(j)
    stats = srv.run()
    assert len(srv.finished) == len(jobs) and srv.used == 0 and not srv.active
    assert max(peak) > max(j.footprint() for j in jobs)   # several jobs did overlap
    assert stats.node_updates == sum(j.node_updates for j in jobs)
    assert all(j.latency is not None and j.latency > 0 for j in jobs)
    for j in jobs:
        with P.Lattice(j.params, stream) as L:
            L.init_rho_u(j.rho, j.ux, j.uy)
            L.step(j.nsteps)
            r, _, _ = L.moments()
        err = float(np.abs(r - j.rho_out).max() / np.abs(r).max())
        assert err < 1e-5, (j.id, err)
