#!/usr/bin/env python
"""Throughput of the fused CTU lattice Boltzmann step on GB300.

Workload (default): the sheared cavitating bubble at the paper's largest
size -- 6144 x 6144 nodes, FP32 shifted storage, CTU2 with the MC limiter,
T = 0.8, tau = 1e-2, kappa = 1e-4, dt = 1e-4, ds = 1/256, sheared walls at
gamma_dot dt = 5e-6 (u_w = 0.6), a tanh vapour seed of radius 26 nodes at
rho_V = 0.23967 in liquid at rho_ext = 1.90, linear initial shear profile.
One "step" = one fused kernel launch advancing all 6144^2 nodes by dt.

Metric: GLUPS = 1e9 node updates per second (one node update = all 16 f_k
of one node advanced one step).  Inputs (2 x 2.25 GiB) exceed L2 (129 MB),
so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank advances its own independent lattice
(replicas; the step has no exchange), timings are max-reduced.

The JSON line adds to the common fields: `roofline` (HBM: algorithmic bytes
per step / step time against MEASURED_PEAKS.json `hbm_gbs`, with the DRAM
traffic of the committed ncu capture of this kernel source), `issue_roofline`
and `fp32_roofline` (instructions and FP32 flops per node update from the
committed capture, against the peaks the library measures on the device with
lbm_measure_peaks), `e2e` (the same metric through the C ABI with pinned host
buffers, copies inside the timed region; median of seven runs, with its phase
times), `cpu_baseline` (the FP64 oracle on
the host cores and on one thread), `clocks`, `config.launch` (the launch
geometry lbm_tune chose before the warm-up, or --row-block's), `runs` (five
more device-resident regions of >= 1 s: GLUPS of each, median, spread) and
`server` (--server NJOBS, default 24: the sweep-server job mix through the
native batch server against the same jobs one at a time -- capacity with every
job submitted at once, then p50/p99 latency and throughput under Poisson
arrivals at twice the serial capacity).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "sheared-bubble-6144": dict(L=6144, T=0.8, tau=1e-2, rho_ext=1.90, rho_v=0.23967, R=26.0,
                                W=4.0, shear_dt=5e-6, walls=True, precision="fp32"),
    # the same physics on a 2048^2 lattice (2 x 268 MB), small enough for ncu captures
    "sheared-bubble-2048": dict(L=2048, T=0.8, tau=1e-2, rho_ext=1.90, rho_v=0.23967, R=26.0,
                                W=4.0, shear_dt=5e-6, walls=True, precision="fp32"),
    # FP16 shifted storage of the same workload: half the bytes per node update
    "sheared-bubble-6144-fp16": dict(L=6144, T=0.8, tau=1e-2, rho_ext=1.90, rho_v=0.23967, R=26.0,
                                     W=4.0, shear_dt=5e-6, walls=True, precision="fp16"),
    "quiescent-bubble-4096": dict(L=4096, T=0.9, tau=1e-3, rho_ext=1.58, rho_v=0.425742, R=20.0,
                                  W=4.0, shear_dt=0.0, walls=False, precision="fp32",
                                  reservoir=True),
    "spinodal-1024-fp64": dict(L=1024, T=0.9, tau=1e-3, rho_ext=1.0, rho_v=1.0, R=0.0, W=0.0,
                               shear_dt=0.0, walls=False, precision="fp64"),
}
METRIC = "GLUPS (16-vel CTU node updates/s) & % HBM roofline"
DT, DS = 1e-4, 1.0 / 256.0


def lib_params(P, w):
    L = w["L"]
    p = P.Params(Lx=L, Ly=L, T=w["T"], tau=w["tau"], dt=DT, ds=DS, rho_ext=w["rho_ext"],
                 precision={"fp32": P.LBM_FP32_SHIFTED, "fp16": P.LBM_FP16_SHIFTED,
                            "fp64": P.LBM_FP64}[w["precision"]],
                 rho_ref=w["rho_ext"])
    if w["walls"]:
        p.boundary = P.LBM_BC_SHEAR_WALLS
        p.shear_rate = w["shear_dt"] / DT
    if w.get("reservoir"):
        p.reservoir = 1
    return p


def initial_fields(w, Lx, Ly):
    import synth
    if w["R"] > 0:
        rho, ux, uy = synth.bubble(Lx, Ly, w["rho_ext"], w["rho_v"], w["R"], w["W"])
    else:
        rho, ux, uy = synth.noisy_uniform(Lx, Ly, 1.0, 1e-2, seed=1)
    if w["walls"]:
        uw = w["shear_dt"] / DT * Ly * DS / 2.0
        ux = synth.linear_shear(Lx, Ly, uw)
    return rho, ux, uy


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("lbm_kernels.cuh", "step_kernel_body.cuh", "step_select.cuh", "step_fp32.cu",
                  "step_fp64.cu", "step_fp16.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1802_01272_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


E2E_REPS = 7  # repetitions of the end-to-end region (median reported)
RUNS, RUN_S = 5, 1.0  # repeated device-resident regions (median and spread reported)
SERVER_LOAD = 2.0      # offered load of the server comparison, x the serial capacity
U_WALL_MAX = 0.5       # server jobs: wall speed cap (Mach ~0.3 in the liquid)


def ncu_record(workload):
    """The committed ncu summary of the step kernel for this workload, if it was
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    e = json.load(open(path)).get(workload)
    if not e or e.get("kernel_source_hash") != kernel_source_hash():
        return None
    return e


def ncu_traffic(workload):
    """DRAM bytes per launch of the step kernel (committed ncu summary) or None."""
    e = ncu_record(workload)
    return None if e is None else float(e["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, seconds=15.0):
    """The FP64 oracle on the host cores, on a bounded sample of the same
    workload: a 192 x 192 window of the initial state, same physics and
    boundaries, stepped until ~`seconds` of CPU work."""
    import oracle as O
    O.build()
    n = 192
    Lx = Ly = w["L"]
    rho, ux, uy = initial_fields(w, Lx, Ly)
    cx, cy = Lx // 2 - n // 2, Ly // 2 - n // 2 if not w["walls"] else 0
    sl = (slice(cy, cy + n), slice(cx, cx + n))
    op = O.Params(Lx=n, Ly=n, T=w["T"], tau=w["tau"], dt=DT, ds=DS, rho_ext=w["rho_ext"],
                  boundary=O.BC_SHEAR_WALLS if w["walls"] else O.BC_PERIODIC,
                  shear_rate=w["shear_dt"] / DT if w["walls"] else 0.0)
    f = O.init_feq(op, rho[sl].copy(), ux[sl].copy(), uy[sl].copy())
    O.step(op, f, 1)  # warm-up
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        f = O.step(op, f, 2)
        steps += 2
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n * n * steps / dt / 1e9, "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n}x{n} window of the {w['L']}^2 workload, FP64 oracle, {steps} steps, "
                      f"{dt:.1f} s"}


def cpu_baseline_single_thread(workload, seconds=5.0):
    """The same oracle sample on one host thread (a child process started
    with OMP_NUM_THREADS=1, since the oracle's thread count is fixed at load)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--workload", workload,
                          "--cpu-baseline-only", str(seconds)], env=env, capture_output=True,
                         text=True, timeout=600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def server_jobs(P, S, njobs, step_scale, seed=4, rate_hz=None):
    """Config 5's job mix: lattices L^2, L in {256, 512, 1024, 2048}; T ~ U[0.75, 0.98];
    shear rate from Ca ~ U[0, 0.4] (Ca = mu_L gamma_dot R / sigma with the seed
    radius R, mu_L = rho_L T tau), with the wall speed u_w = gamma_dot L ds / 2
    capped at U_WALL_MAX (on the large lattices Ca = 0.4 at R = 20 nodes would
    need walls faster than sound); a tanh vapour seed (R = 20, W = 4) in liquid
    at rho_L(T); steps ~ U{5000..20000} x step_scale; Poisson arrivals."""
    import numpy as np
    import synth
    from paper_1802_01272_gb300 import eos
    rng = np.random.default_rng(seed)
    jobs, t = [], 0.0
    for i in range(njobs):
        L = int(rng.choice([256, 512, 1024, 2048]))
        T = float(rng.uniform(0.75, 0.98))
        ca = float(rng.uniform(0.0, 0.4))
        rl, rv = eos.coexistence(T)
        sigma = eos.interface_tension(T, 1e-4)
        tau = 1e-2
        gdot = min(ca * sigma / (rl * T * tau * 20 * DS), 2.0 * U_WALL_MAX / (L * DS))
        p = P.Params(Lx=L, Ly=L, T=T, tau=tau, dt=DT, ds=DS, rho_ext=rl, rho_ref=rl,
                     boundary=P.LBM_BC_SHEAR_WALLS if gdot > 0 else P.LBM_BC_PERIODIC,
                     shear_rate=gdot)
        rho, ux, uy = synth.bubble(L, L, rl, rv, 20.0, 4.0)
        if gdot > 0:
            ux = synth.linear_shear(L, L, gdot * L * DS / 2)
        nsteps = max(10, int(int(rng.integers(5000, 20001)) * step_scale))
        jobs.append(S.Job(params=p, rho=rho, ux=ux, uy=uy, nsteps=nsteps, arrival=t,
                          diag_threshold=0.5 * (rl + rv)))
        t += float(rng.exponential(1.0 / rate_hz)) if rate_hz else 0.0
    return jobs


def run_server_bench(P, stream, njobs, step_scale):
    """Continuous batching vs the same jobs one at a time (same GPU, same jobs).
    Capacity: every job submitted at t = 0 (GLUPS = work / makespan).  Then
    Poisson arrivals offered at LOAD x the serial capacity, for the latencies
    (p50, p99 of finish - arrival) and the throughput under that load."""
    from paper_1802_01272_gb300 import server as S
    jobs = server_jobs(P, S, njobs, step_scale)
    work = sum(j.node_updates for j in jobs)
    cap_serial = S.run_serial(server_jobs(P, S, njobs, step_scale), stream)
    with S.BatchServer(mem_budget_bytes=int(64e9), chunk=100) as srv:
        cap_batched = S.run_jobs(srv, server_jobs(P, S, njobs, step_scale))
    rate_hz = SERVER_LOAD * cap_serial.glups * 1e9 / (work / njobs)
    jobs = server_jobs(P, S, njobs, step_scale, rate_hz=rate_hz)
    with S.BatchServer(mem_budget_bytes=int(64e9), chunk=100) as srv:
        st = S.run_jobs(srv, jobs)
    ss = S.run_serial(server_jobs(P, S, njobs, step_scale, rate_hz=rate_hz), stream)
    return {"jobs": njobs, "steps_scale": step_scale, "node_updates": work,
            "capacity_glups": {"batched": cap_batched.glups, "serial": cap_serial.glups,
                               "note": "all jobs submitted at t = 0; work / makespan"},
            "offered_load": f"Poisson arrivals at {SERVER_LOAD} x the serial capacity",
            "batched": {"glups": st.glups, "p50_s": st.pct(50), "p99_s": st.pct(99),
                        "makespan_s": st.makespan, "launches": st.launches,
                        "server": "native lbm_batch_* (C++ worker thread)"},
            "serial": {"glups": ss.glups, "p50_s": ss.pct(50), "p99_s": ss.pct(99),
                       "makespan_s": ss.makespan}}


def make_sync(dist, device):
    """The timing protocol's helpers for one rank: barrier() synchronises the
    device on both sides of a process-group barrier (a no-op group of one when
    dist is None); max_over_ranks(x) returns the largest x over all ranks."""
    import torch

    def sync():
        if device.type == "cuda":
            torch.cuda.synchronize(device)

    def barrier():
        sync()
        if dist is not None:
            dist.barrier()
            sync()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return barrier, max_over_ranks


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    cb = cpu_baseline(w, seconds=max(5.0, min(20.0, 3.0 * args.steps)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "GLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "lattice": w["L"], "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sheared-bubble-6144", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch geometry")
    ap.add_argument("--row-block", type=int, default=0,
                    help="fix the row-block height (as many CTAs per SM as fit) instead of tuning")
    ap.add_argument("--cpu-baseline-only", type=float, default=None, metavar="SECONDS",
                    help="print the oracle's host-core sample for this workload and exit")
    ap.add_argument("--no-repeats", action="store_true",
                    help="skip the repeated >= 1 s regions (profiling runs)")
    ap.add_argument("--server", type=int, default=24, metavar="NJOBS",
                    help="sweep-server comparison over NJOBS config-5 jobs (0: off)")
    ap.add_argument("--server-step-scale", type=float, default=0.05)
    ap.add_argument("--ctu-order", type=int, default=None, help="override the scheme (profiling)")
    ap.add_argument("--limiter", type=int, default=None, help="override the limiter (profiling)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.cpu_baseline_only is not None:
        print(json.dumps(cpu_baseline(w, seconds=args.cpu_baseline_only)), flush=True)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import numpy as np
    import torch
    import paper_1802_01272_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    p = lib_params(P, w)
    if args.ctu_order is not None:
        p.ctu_order = args.ctu_order
    if args.limiter is not None:
        p.limiter = args.limiter
    rho, ux, uy = initial_fields(w, p.Lx, p.Ly)
    nodes = p.Lx * p.Ly
    elem = {P.LBM_FP32_SHIFTED: 4, P.LBM_FP16_SHIFTED: 2}.get(p.precision, 8)

    barrier, max_over_ranks = make_sync(dist, torch.device("cuda", local))

    # ---------------- device-resident throughput
    L = P.Lattice(p, stream)
    d_rho, d_ux, d_uy = (torch.from_numpy(x).cuda() for x in (rho, ux, uy))
    L.init_rho_u_device(d_rho, d_ux, d_uy)
    # launch geometry from the library's autotuner (its trial steps are part of
    # the untimed warm-up)
    if args.row_block:
        launch = L.set_launch(args.row_block)
    else:
        launch = L.tune(3) if not args.no_tune else L.kernel_info()
    L.step(args.warmup)
    L.sync()
    # measured compute peaks for the issue and FP32 rooflines (untimed)
    from paper_1802_01272_gb300.binding import measure_peaks
    peaks = measure_peaks(stream)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    L.step(args.steps)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    # repeats: RUNS more regions of at least RUN_S seconds each (at least K
    # steps), for the median and spread of the step time
    per_step = ms / args.steps
    rep_steps = max(args.steps, int(RUN_S * 1e3 / max(per_step, 1e-6)) + 1)
    run_ms = []
    for _ in range(RUNS if not args.no_repeats else 0):
        barrier()
        e0.record(stream)
        L.step(rep_steps)
        e1.record(stream)
        barrier()
        run_ms.append(max_over_ranks(e0.elapsed_time(e1)))
    clk = clocks.stop()
    L.sync()
    ms = max_over_ranks(ms)
    ms_per_step = ms / args.steps
    value = world * nodes * args.steps / (ms * 1e-3) / 1e9
    rep_glups = [world * nodes * rep_steps / (m * 1e-3) / 1e9 for m in run_ms]

    # roofline of the step kernel: the only kernel in the timed region
    peak, peak_kind = load_peaks()
    alg_bytes = 2 * 16 * elem * nodes
    achieved = alg_bytes / (ms_per_step * 1e-3) / 1e9
    traffic = ncu_traffic(args.workload)
    # the step is bound by instruction issue, not HBM: GB300 issues
    # 4 warp-instructions per clock per SM; the instructions per node update
    # come from the committed ncu capture of this kernel source
    rec = ncu_record(args.workload)
    issue_roof = fp32_roof = None
    if rec and rec.get("thread_instructions_per_node"):
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        ipn = float(rec["thread_instructions_per_node"])
        ach = ipn * value / world * 1e9 / 1e12
        derived = nsm * 4 * 32 * mhz * 1e6 / 1e12
        pk = peaks["issue_rate"] * 32 / 1e12 if peaks else derived
        issue_roof = {"bound": "alu", "instructions_per_node": ipn, "achieved": ach, "peak": pk,
                      "unit": "T thread-instructions/s", "frac": ach / pk,
                      "peak_source": "measured (lbm_measure_peaks: FP32 min3 + add chains)"
                      if peaks else "derived", "peak_derived":
                      derived, "peak_derived_source":
                      f"{nsm} SMs x 4 issue slots x 32 lanes x {mhz:.0f} MHz"}
    if rec and rec.get("fp32_flops_per_node") and peaks:
        fpn = float(rec["fp32_flops_per_node"])
        ach = fpn * value / world * 1e9 / 1e12
        pk = peaks["fp32_flops"] / 1e12
        fp32_roof = {"bound": "fp32", "flops_per_node": fpn, "achieved": ach, "peak": pk,
                     "unit": "TFLOP/s", "frac": ach / pk,
                     "peak_source": "measured (lbm_measure_peaks: FFMA chains)"}

    # ---------------- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = [torch.empty(p.Ly, p.Lx, dtype=torch.float64).pin_memory() for _ in range(6)]
        for t, x in zip(pin[:3], (rho, ux, uy)):
            t.numpy()[...] = x
        hr, hx, hy = (t.numpy() for t in pin[:3])
        orho, oux, ouy = (t.numpy() for t in pin[3:])
        E = P.Lattice(p, stream)
        if args.row_block:
            E.set_launch(args.row_block)
        elif not args.no_tune:
            E.tune(3)                    # untimed, like the warm-up
        thr = 0.5 * (w["rho_ext"] + w["rho_v"])
        E.init_rho_u(hr, hx, hy)
        E.step_diag(2, thr)
        E.moments(out=(orho, oux, ouy))  # first device access of the pinned outputs
        # the region runs E2E_REPS times; host transfers share the host's memory
        # with other tenants, so the median run is reported, with its phases
        runs = []
        for _ in range(E2E_REPS):
            barrier()
            t0 = time.perf_counter()
            E.init_rho_u(hr, hx, hy)
            t1 = time.perf_counter()
            for _ in range(args.steps):
                E.step_diag(1, thr)      # one step, its diagnostics record read back
            t2 = time.perf_counter()
            E.moments(out=(orho, oux, ouy))
            barrier()
            t3 = time.perf_counter()
            runs.append((max_over_ranks(t3 - t0), t1 - t0, t2 - t1, t3 - t2))
        E.close()
        runs.sort()
        te, ti, ts, to = runs[len(runs) // 2]
        diag_bytes = 17 * 8
        e2e = {"value": world * nodes * args.steps / te / 1e9, "unit": "GLUPS",
               "h2d_bytes_per_step": int(3 * 8 * nodes / args.steps),
               "d2h_bytes_per_step": int(diag_bytes + 3 * 8 * nodes / args.steps),
               "region": "init_rho_u from pinned host + per step lbm_step_diag(1) (diagnostics "
                         "record reduced in the step, read back) + final lbm_moments to host",
               "runs": len(runs), "run_values": [world * nodes * args.steps / r[0] / 1e9 for r in runs],
               "phase_ms": {"h2d_and_init": ti * 1e3, "steps": ts * 1e3, "d2h": to * 1e3}}
    L.close()

    srv = None
    if args.server and world == 1:
        srv = run_server_bench(P, stream, args.server, args.server_step_scale)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w)
        one = cpu_baseline_single_thread(args.workload)
        cb["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if elem == 8 else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "lattice": [p.Lx, p.Ly],
                       "storage": {4: "fp32 shifted (f - w rho_ref)",
                                   2: "fp16 shifted (f - w rho_ref), fp32 arithmetic"}.get(elem, "fp64"),
                       "scheme": {1: "CTU1", 2: "CTU2"}[p.ctu_order] +
                                 {0: " + MC limiter", 1: " (Psi = 0)", 2: " (Psi = 1)"}[p.limiter]
                                 if p.ctu_order == 2 else "CTU1", "T": p.T, "tau": p.tau,
                       "boundary": "shear walls" if w["walls"] else "periodic",
                       "l2": "inputs 2x%.2f GiB > L2, no flush" % (16 * elem * nodes / 2**30),
                       "parallelism": f"replicas x{world}",
                       "launch": {k: launch[k] for k in ("grid", "row_block", "tensor_copies")}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                         if peak_kind == "measured" else "fallback 6.8 TB/s",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "runs": {"steps_each": rep_steps, "glups": rep_glups,
                     "median": statistics.median(rep_glups) if rep_glups else None,
                     "spread": (max(rep_glups) - min(rep_glups)) / statistics.median(rep_glups)
                     if rep_glups else None},
            "issue_roofline": issue_roof,
            "fp32_roofline": fp32_roof,
            "gpu_launches": args.steps,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cb,
        }
        if srv is not None:
            line["server"] = srv
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
