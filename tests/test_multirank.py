"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).  The path shards over
independent volume pairs (replicas): each rank solves its own pair, the only collective is the
max of the per-rank times, and the job's throughput is the units of all ranks over that max.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        w, r, local = bench.rank_env()
        seconds = 1.0 + 0.5 * r                  # rank 1 is the slower one
        slowest = bench.max_over_ranks(seconds, dist, torch.device("cpu"))
        value = bench.job_throughput(w, 3, slowest)
        seeds = [None] * w
        dist.all_gather_object(seeds, bench.rank_seed("tiny", r))
        out.put((r, w, local, slowest, value, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_distinct_pairs():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, slowest, value, seeds) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert slowest == 1.5                     # the max over ranks, on every rank
        assert value == pytest.approx(2 * 3 / 1.5)
        assert seeds[0] != seeds[1]               # each rank solves its own pair


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.rank_env() == (1, 0, 0)
        assert bench.max_over_ranks(2.5, None, None) == 2.5
        assert bench.job_throughput(1, 10, 2.0) == 5.0
    finally:
        os.environ.update(env)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    """`bench.py --impl reference` launched on 2 ranks: rank 0 times the oracle and prints the
    JSON line, rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "pairs/s"
    assert d["cpu_baseline"]["kind"] == "oracle"
