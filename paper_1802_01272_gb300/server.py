"""Continuous-batching sweep server for many CTU lattice Boltzmann jobs.

Parameter sweeps (phase diagrams over T, shear-rate sweeps over the
capillary number) are many independent lattices.  The server keeps every
admitted job's lattice resident in device memory and advances all active
jobs together: each tick is one `lbm_step_many` call, i.e. one fused launch
per step covering every compatible lattice, so small lattices that could not
fill the GPU alone share it.  Jobs that arrive while others run are admitted
as soon as their device-memory footprint fits the budget, and a finished job
releases its memory at once (continuous batching, not a queue).

Each job's result is the one it would have alone, to FP32 rounding (the
batched launch performs the same per-node operations), which the tests check.

The scheduling loop runs on the calling thread (`run`), with arrivals given
as timestamps; `submit` may also be called from other threads.
"""
from __future__ import annotations

import heapq
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from .binding import LBM_FP64, Lattice, Params, step_many


@dataclass
class Job:
    params: Params
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    nsteps: int
    arrival: float = 0.0            # seconds after the server starts
    diag_threshold: float | None = None
    id: int = -1
    # filled by the server
    admitted: float | None = None
    finished: float | None = None
    diag: dict | None = None
    rho_out: np.ndarray | None = None
    done_steps: int = 0
    keep_rho: bool = False

    def footprint(self) -> int:
        """Device bytes of the job: two ping-pong buffers of 16 planes."""
        elem = 8 if self.params.precision == LBM_FP64 else 4
        return 2 * 16 * elem * self.params.Lx * self.params.Ly + 3 * 8 * self.params.Lx * self.params.Ly

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

    @property
    def glups(self) -> float:
        return self.node_updates / self.makespan / 1e9

    def pct(self, q) -> float:
        return float(np.percentile(self.latencies, q)) if self.latencies else float("nan")


class SweepServer:
    """Admits jobs by device-memory footprint and advances all active jobs in
    batched launches of `chunk` steps (fewer when a job is about to finish)."""

    def __init__(self, mem_budget_bytes: int, stream=None, chunk: int = 200,
                 max_active: int = 64):
        self.budget = int(mem_budget_bytes)
        self.stream = stream
        self.chunk = int(chunk)
        self.max_active = int(max_active)
        self._lock = threading.Lock()
        self._pending: list = []     # heap of (arrival, id, job)
        self._next_id = 0
        self.active: list = []       # (job, lattice)
        self.used = 0
        self.finished: list = []

    def submit(self, job: Job) -> int:
        if job.footprint() > self.budget:
            raise ValueError(f"job needs {job.footprint()} B, above the budget {self.budget} B")
        with self._lock:
            job.id = self._next_id
            self._next_id += 1
            heapq.heappush(self._pending, (job.arrival, job.id, job))
        return job.id

    def _admit(self, now: float):
        with self._lock:
            while (self._pending and self._pending[0][0] <= now
                   and len(self.active) < self.max_active
                   and self.used + self._pending[0][2].footprint() <= self.budget):
                _, _, job = heapq.heappop(self._pending)
                L = Lattice(job.params, self.stream)
                L.init_rho_u(job.rho, job.ux, job.uy)
                job.admitted = now
                self.used += job.footprint()
                self.active.append((job, L))

    def _retire(self, now_fn):
        keep = []
        for job, L in self.active:
            if job.done_steps >= job.nsteps:
                if job.diag_threshold is not None:
                    job.diag = L.diagnostics(job.diag_threshold)
                if job.keep_rho:
                    job.rho_out = L.moments()[0]
                else:
                    L.sync()
                job.finished = now_fn()
                self.used -= job.footprint()
                L.close()
                self.finished.append(job)
            else:
                keep.append((job, L))
        self.active = keep

    def run(self, clock=time.perf_counter) -> ServerStats:
        """Serve until every submitted job is finished; arrivals are relative
        to the start of this call."""
        t0 = clock()
        now = lambda: clock() - t0
        total = 0
        while True:
            self._admit(now())
            if not self.active:
                with self._lock:
                    if not self._pending:
                        break
                    wait = self._pending[0][0] - now()
                if wait > 0:
                    time.sleep(min(wait, 0.01))
                continue
            k = min(self.chunk, min(j.nsteps - j.done_steps for j, _ in self.active))
            step_many([L for _, L in self.active], k)
            for j, _ in self.active:
                j.done_steps += k
                total += j.params.Lx * j.params.Ly * k
            self._retire(now)
        return ServerStats(makespan=now(), node_updates=total,
                           latencies=[j.latency for j in self.finished])


def run_serial(jobs, stream=None, clock=time.perf_counter) -> ServerStats:
    """Baseline: the same jobs one after another through lbm_step (FIFO by
    arrival), each alone on the GPU."""
    t0 = clock()
    total = 0
    lat = []
    for job in sorted(jobs, key=lambda j: j.arrival):
        while clock() - t0 < job.arrival:
            time.sleep(min(job.arrival - (clock() - t0), 0.01))
        with Lattice(job.params, stream) as L:
            L.init_rho_u(job.rho, job.ux, job.uy)
            L.step(job.nsteps)
            if job.diag_threshold is not None:
                job.diag = L.diagnostics(job.diag_threshold)
            else:
                L.sync()
        job.finished = clock() - t0
        lat.append(job.latency)
        total += job.node_updates
    return ServerStats(makespan=clock() - t0, node_updates=total, latencies=lat)
