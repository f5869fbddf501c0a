"""Host logic of bench.py without a GPU: the multi-rank timing helpers on two
gloo ranks, and the reference arm (the FP64 oracle on the host cores)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    barrier, max_over_ranks = bench.make_sync(dist, torch.device("cpu"))
    barrier()
    m = max_over_ranks(1.5 + rank)
    barrier()
    dist.destroy_process_group()
    out.put((rank, m))


def test_max_over_ranks_and_barrier_on_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]


def test_single_rank_helpers_are_identity():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    barrier, max_over_ranks = bench.make_sync(None, torch.device("cpu"))
    barrier()
    assert max_over_ranks(3.25) == 3.25


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "GLUPS"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    # under torchrun, ranks other than 0 exit at once without output
    env.update(RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_single_thread_oracle_sample():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.cpu_baseline_single_thread("sheared-bubble-2048", seconds=1.0)
    assert one["kind"] == "oracle" and one["cores"] == 1 and one["value"] > 0


def test_server_job_mix_follows_config5_with_capped_walls():
    """The sweep-server job mix (config 5): lattice sizes from {256, 512, 1024,
    2048}^2, T in [0.75, 0.98], steps in 5000..20000 x the scale, Poisson
    arrival times increasing; wall speeds capped at bench.U_WALL_MAX (below the
    method's stability limit in uniform flow, test_oracle_stability)."""
    import bench
    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300 import server as S
    jobs = bench.server_jobs(P, S, 24, 0.05, rate_hz=10.0)
    assert {j.params.Lx for j in jobs} <= {256, 512, 1024, 2048}
    assert all(j.params.Lx == j.params.Ly for j in jobs)
    assert all(0.75 <= j.params.T <= 0.98 for j in jobs)
    assert all(250 <= j.nsteps <= 1000 for j in jobs)
    uw = [j.params.shear_rate * j.params.Ly * j.params.ds / 2 for j in jobs]
    assert max(uw) <= bench.U_WALL_MAX + 1e-12 and max(uw) > 0.0
    arr = [j.arrival for j in jobs]
    assert arr[0] == 0.0 and all(b > a for a, b in zip(arr, arr[1:]))
