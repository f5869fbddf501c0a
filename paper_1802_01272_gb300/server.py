"""Continuous-batching sweep server for many CTU lattice Boltzmann jobs.

Parameter sweeps (phase diagrams over T, shear-rate sweeps over the
capillary number) are many independent lattices.  `BatchServer` wraps the
library's native server (lbm_batch_* in include/ctulbm.h): a C++ worker
thread admits jobs in submission order while their device footprint fits the
budget, advances resident jobs together (one batched launch per step, so
small lattices that could not fill the GPU alone share it; each tick the jobs
with the least work left, as many as fill the GPU), records diagnostics, and
frees a finished job's memory at once.  This module only
marshals jobs in and results out; `run_jobs` replays an arrival process and
`run_serial` is the one-job-at-a-time baseline.

Each job's result is the one it would have alone, to FP32 rounding (the
batched launch performs the same per-node operations), which the tests check.
"""
from __future__ import annotations

import ctypes as C
import time
from dataclasses import dataclass, field

import numpy as np

from .binding import (LBM_FP16_SHIFTED, LBM_FP64, LBM_JOB_DONE, LBM_JOB_FAILED, Lattice, LBMError,
                      Params, _check, _host, _stream_ptr, lbm_batch_info, lbm_diag, lbm_job_result,
                      lib)


@dataclass
class Job:
    params: Params
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    nsteps: int
    arrival: float = 0.0            # seconds after the start of run_jobs / run_serial
    diag_threshold: float | None = None
    diag_every: int = 0             # 0: a diagnostics record at the end only
    keep_rho: bool = False
    id: int = -1
    # filled in
    submitted: float | None = None  # wall clock of the submission (run_jobs clock)
    finished: float | None = None
    diag: dict | None = None
    rho_out: np.ndarray | None = None
    status: int = -1
    error: int = 0

    def footprint(self) -> int:
        """Device bytes the server reserves for the job (as the library counts)."""
        elem = {LBM_FP64: 8, LBM_FP16_SHIFTED: 2}.get(self.params.precision, 4)
        n = self.params.Lx * self.params.Ly
        return 32 * elem * n + 24 * n + 4096

    @property
    def node_updates(self) -> int:
        return self.params.Lx * self.params.Ly * self.nsteps

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival


@dataclass
class ServerStats:
    makespan: float
    node_updates: int
    latencies: list = field(default_factory=list)
    launches: int = 0

    @property
    def glups(self) -> float:
        return self.node_updates / self.makespan / 1e9

    def pct(self, q) -> float:
        return float(np.percentile(self.latencies, q)) if self.latencies else float("nan")


def _diag_dict(d: lbm_diag) -> dict:
    return {n: getattr(d, n) for n, _ in lbm_diag._fields_}


class BatchServer:
    """The library's continuous-batching server (lbm_batch_*)."""

    def __init__(self, mem_budget_bytes: int, chunk: int = 100, stream=None):
        self._b = C.c_void_p()
        _check(lib().lbm_batch_create(int(mem_budget_bytes), int(chunk), _stream_ptr(stream),
                                      C.byref(self._b)), "lbm_batch_create")

    def submit(self, job: Job) -> int:
        shape = (job.params.Ly, job.params.Lx)
        a = [_host(x, shape) for x in (job.rho, job.ux, job.uy)]
        thr = job.diag_threshold if job.diag_threshold is not None else 0.0
        jid = lib().lbm_batch_submit(self._b, C.byref(job.params.c()),
                                     *[x.ctypes.data for x in a], int(job.nsteps),
                                     int(job.diag_every), thr)
        if jid < 0:
            raise LBMError(int(jid), "lbm_batch_submit")
        job.id = int(jid)
        return job.id

    def poll(self, job_id: int) -> lbm_job_result:
        r = lbm_job_result()
        _check(lib().lbm_batch_poll(self._b, job_id, C.byref(r)), "lbm_batch_poll")
        return r

    def wait(self, job_id: int = -1, timeout: float | None = None) -> None:
        _check(lib().lbm_batch_wait(self._b, job_id, -1.0 if timeout is None else timeout, None),
               "lbm_batch_wait")

    def fetch(self, job: Job) -> None:
        """Fill job.diag, job.status and (if job.keep_rho) job.rho_out from a
        finished job; the server then drops the job's final fields."""
        r = self.poll(job.id)
        job.status, job.error = r.status, r.error
        job.diag = _diag_dict(r.diag) if r.diag_step >= 0 else None
        if r.status == LBM_JOB_DONE:
            rho = np.empty((job.params.Ly, job.params.Lx)) if job.keep_rho else None
            _check(lib().lbm_batch_fetch(self._b, job.id,
                                         rho.ctypes.data if rho is not None else None, None, None),
                   "lbm_batch_fetch")
            job.rho_out = rho

    def info(self) -> dict:
        i = lbm_batch_info()
        _check(lib().lbm_batch_get_info(self._b, C.byref(i)), "lbm_batch_get_info")
        return {n: getattr(i, n) for n, _ in lbm_batch_info._fields_}

    def close(self):
        if self._b:
            lib().lbm_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_jobs(server: BatchServer, jobs, clock=time.perf_counter) -> ServerStats:
    """Submit each job at its arrival time (relative to this call), wait for
    all, collect results.  Latency = finish - arrival, with the finish time
    taken from the server's own record of the job's end."""
    order = sorted(jobs, key=lambda j: j.arrival)
    t0 = clock()
    offsets = []
    for j in order:
        while clock() - t0 < j.arrival:
            time.sleep(min(j.arrival - (clock() - t0), 0.005))
        server.submit(j)
        r = server.poll(j.id)
        j.submitted = clock() - t0
        offsets.append(j.submitted - r.t_submit)    # run_jobs clock - server clock
    server.wait(-1)
    makespan = clock() - t0
    off = float(np.median(offsets))
    for j in order:
        r = server.poll(j.id)
        j.finished = r.t_finish + off
        server.fetch(j)
        if j.status == LBM_JOB_FAILED:
            raise LBMError(j.error, f"batch job {j.id}")
    info = server.info()
    return ServerStats(makespan=makespan, node_updates=sum(j.node_updates for j in order),
                       latencies=[j.latency for j in order], launches=info["launches"])


def run_serial(jobs, stream=None, clock=time.perf_counter) -> ServerStats:
    """Baseline: the same jobs one after another through lbm_step (FIFO by
    arrival), each alone on the GPU."""
    t0 = clock()
    total = 0
    lat = []
    for job in sorted(jobs, key=lambda j: j.arrival):
        while clock() - t0 < job.arrival:
            time.sleep(min(job.arrival - (clock() - t0), 0.005))
        with Lattice(job.params, stream) as L:
            L.init_rho_u(job.rho, job.ux, job.uy)
            L.step(job.nsteps)
            if job.diag_threshold is not None:
                job.diag = L.diagnostics(job.diag_threshold)
            if job.keep_rho:
                job.rho_out = L.moments()[0]
            else:
                L.sync()
        job.finished = clock() - t0
        lat.append(job.latency)
        total += job.node_updates
    return ServerStats(makespan=clock() - t0, node_updates=total, latencies=lat)
