"""The native continuous-batching server (lbm_batch_*): jobs admitted in
submission order by device footprint, advanced together, each result the one
it has alone (to FP32 rounding), diagnostics recorded on schedule."""
import threading
import time

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
        prec = P.LBM_FP64 if i == 3 else P.LBM_FP32_SHIFTED      # one job steps on its own
        lp = P.Params(Lx=L, Ly=L, T=T, tau=1e-3, rho_ext=1.6, rho_ref=1.6, precision=prec)
        rho, ux, uy = synth.bubble(L, L, 1.6, 0.5, R=L / 6, W=2)
        jobs.append(S.Job(params=lp, rho=rho, ux=ux, uy=uy, nsteps=int(rng.integers(100, 400)),
                          arrival=0.002 * i, diag_threshold=1.0, diag_every=50, keep_rho=True))
    return jobs


def test_server_results_equal_alone_and_admission_respects_budget():
    import torch
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import server as S
    stream = torch.cuda.current_stream()
    jobs = make_jobs(P, S)
    budget = 3 * max(j.footprint() for j in jobs)        # at most ~3 resident at once
    peak, stop = [], threading.Event()
    with S.BatchServer(budget, chunk=64) as srv:
        def watch():
            while not stop.is_set():
                peak.append(srv.info()["used_bytes"])
                time.sleep(0.0005)
        th = threading.Thread(target=watch)
        th.start()
        stats = S.run_jobs(srv, jobs)
        stop.set()
        th.join()
        info = srv.info()
    assert info["done"] == len(jobs) and info["failed"] == 0 and info["used_bytes"] == 0
    assert max(peak) <= budget
    assert max(peak) > max(j.footprint() for j in jobs)   # several jobs did overlap
    assert info["node_updates"] == stats.node_updates == sum(j.node_updates for j in jobs)
    assert all(j.latency is not None and j.latency > 0 for j in jobs)
    for j in jobs:
        with P.Lattice(j.params, stream) as L:
            L.init_rho_u(j.rho, j.ux, j.uy)
            L.step(j.nsteps)
            r, _, _ = L.moments()
            d = L.diagnostics(1.0)
        err = float(np.abs(r - j.rho_out).max() / np.abs(r).max())
        tol = 1e-12 if j.params.precision == P.LBM_FP64 else 1e-5
        assert err < tol, (j.id, err)
        assert j.diag is not None and abs(j.diag["mass"] - d["mass"]) / d["mass"] < 1e-6


def test_server_diagnostics_schedule_and_poll():
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import server as S
    lp = P.Params(Lx=128, Ly=96, T=0.85, rho_ref=1.6, rho_ext=1.6)
    rho, ux, uy = synth.bubble(128, 96, 1.6, 0.5, R=16, W=2)
    job = S.Job(params=lp, rho=rho, ux=ux, uy=uy, nsteps=250, diag_threshold=1.0, diag_every=100)
    with S.BatchServer(1 << 30, chunk=1000) as srv:
        srv.submit(job)
        srv.wait(job.id)
        r = srv.poll(job.id)
        assert r.status == P.binding.LBM_JOB_DONE and r.steps_done == 250 and r.diag_step == 250
        assert r.t_submit <= r.t_start <= r.t_finish
        assert srv.info()["launches"] == 3                   # 100 + 100 + 50 steps
        srv.fetch(job)
        with pytest.raises(P.LBMError):                      # final fields already released
            P.binding._check(P.lib().lbm_batch_fetch(srv._b, job.id, None, None, None), "fetch")
        with pytest.raises(P.LBMError):                      # larger than the whole budget
            big = S.Job(params=P.Params(Lx=4096, Ly=4096), rho=np.ones((4096, 4096)),
                        ux=np.zeros((4096, 4096)), uy=np.zeros((4096, 4096)), nsteps=1)
            srv.submit(big)


def test_server_large_jobs_equal_alone_in_the_mix():
    """Jobs of 512^2 .. 1024^2 nodes and 1000 .. 1200 steps, overlapping in the
    server's batched launches (graph launches of 16 steps), each ends where it
    ends alone through lbm_step: the batched kernel runs every node through
    the same arithmetic, so FP32 results agree to rounding (the bar is the
    FP32 accuracy bar, 1e-5; the difference measured is printed) and the FP64
    job, which steps on its own, agrees bit for bit."""
    import torch
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import server as S
    stream = torch.cuda.current_stream()
    spec = [(512, 1000, P.LBM_FP32_SHIFTED), (768, 1200, P.LBM_FP32_SHIFTED),
            (1024, 1000, P.LBM_FP32_SHIFTED), (512, 1100, P.LBM_FP32_SHIFTED),
            (512, 1000, P.LBM_FP64)]
    jobs = []
    for i, (L, n, prec) in enumerate(spec):
        lp = P.Params(Lx=L, Ly=L, T=0.85, tau=1e-3, rho_ext=1.6, rho_ref=1.6, precision=prec)
        rho, ux, uy = synth.bubble(L, L, 1.6, 0.5, R=L / 8, W=3)
        jobs.append(S.Job(params=lp, rho=rho, ux=ux, uy=uy, nsteps=n, arrival=0.01 * i,
                          diag_threshold=1.0, keep_rho=True))
    with S.BatchServer(int(16e9), chunk=400) as srv:
        S.run_jobs(srv, jobs)
        info = srv.info()
    assert info["done"] == len(jobs) and info["failed"] == 0
    for j in jobs:
        with P.Lattice(j.params, stream) as L:
            L.init_rho_u(j.rho, j.ux, j.uy)
            L.step(j.nsteps)
            r, _, _ = L.moments()
        err = float(np.abs(r - j.rho_out).max() / np.abs(r).max())
        print(f"\n{j.params.Lx}^2 x {j.nsteps} steps, precision {j.params.precision}: "
              f"alone vs in the mix {err:.3e}")
        if j.params.precision == P.LBM_FP64:
            assert np.array_equal(r, j.rho_out)
        else:
            assert err < 1e-5
