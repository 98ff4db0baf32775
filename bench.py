"""Throughput benchmark: corrected 3T-shaped volume pairs per second at a fixed GN iteration count.

One step = one full solve of one 144x168x111 (1.25 mm, PE along the 168 axis) synthetic pair:
OT initialisation with blur + 20 Gauss-Newton iterations, each with up to 10 Jacobi-PCG
iterations and an Armijo line search (the paper's default method, Sec. 2.2-2.3.1), inputs
resident in HBM.  L2 is flushed before every timed step (a 256 MiB write, then a 256 MiB read of a
second buffer, so that no dirty line of the flush is left to be written back inside the timed
region); each step is timed with CUDA events on the launching stream and the flush is outside the
events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload 3t]

N > 1 runs under torchrun: every rank solves its own pairs (independent problems, no data-path
collective); the timing is the max over ranks and value = total pairs / that time.
--impl reference times the CPU oracle (the reference arm of this build) on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2403_10706_b300 import phantom as ph  # noqa: E402

METRIC = "corrected 3T-shaped volume pairs/sec (fixed GN iters); eval-kernel HBM GB/s vs peak"
UNIT = "pairs/s"
GN_ITERS = {"3t": 20, "7t": 20, "small": 20, "tiny": 10, "7t_paper": 20}
ALPHA, BETA = 300.0, 1e4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3t", choices=list(GN_ITERS))
    ap.add_argument("--precond", type=int, default=0)
    ap.add_argument("--pcg-path", type=int, default=0,
                    help="0 auto (= 2 when possible), 1 separate kernels, 2 persistent kernel, "
                         "3 persistent one-barrier-per-iteration kernel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 64-pair uneven batch (batched vs sequential solves)")
    ap.add_argument("--no-admm", action="store_true",
                    help="skip the ADMM timing row (e.g. for short profiling runs)")
    ap.add_argument("--no-extra-shapes", action="store_true",
                    help="skip the paper's 7T acquisition size (e.g. for short profiling runs)")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the bf16 / f16 image-storage timing")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def tf32_peak():
    """Dense TF32 tensor TFLOP/s: the measured bf16 burst figure x the nominal TF32/BF16 ratio
    (1.1 / 2.25 PFLOP/s), else the fallback bf16 figure x that ratio."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x 1.1/2.25"
    return 1800.0 * 1.1 / 2.25, "fallback bf16 x 1.1/2.25"


EVAL_SOURCES = ["paper_2403_10706_b300/csrc/k_eval.cu",
                "paper_2403_10706_b300/csrc/eval_march.cuh",
                "paper_2403_10706_b300/csrc/eval_common.cuh",
                "paper_2403_10706_b300/csrc/hysco_internal.cuh"]
PCG_SOURCES = ["paper_2403_10706_b300/csrc/k_pcg_persistent.cu",
               "paper_2403_10706_b300/csrc/pcg_run.cuh",
               "paper_2403_10706_b300/csrc/grid_sync.cuh",
               "paper_2403_10706_b300/csrc/hysco_internal.cuh"]


def _current_profile(profile, sources):
    """Text of a committed ncu summary, or None when the kernel's sources have changed since the
    counters were taken (the summary records a hash of them)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    rec = dict(line.split(":", 1) for line in text.splitlines() if line.startswith("source-sha256:"))
    if rec.get("source-sha256", "").split()[0:1] != [h.hexdigest()[:16]]:
        return None
    return text


def recorded_traffic(profile, sources):
    """DRAM bytes per launch from a committed, current ncu summary (else None)."""
    text = _current_profile(profile, sources)
    if text is None:
        return None
    # the first record is the summary's own kernel (later sections cover its variants)
    for line in text.splitlines():
        if line.startswith("dram-bytes-per-launch:"):
            return int(line.split(":", 1)[1].strip())
    return None


def recorded_warp_instructions(profile, sources):
    """Warp instructions executed per launch (smsp__inst_executed.sum) from a committed, current
    ncu summary (else None)."""
    text = _current_profile(profile, sources)
    if text is None:
        return None
    for line in text.splitlines():
        if line.startswith("| `smsp__inst_executed.sum`"):
            return float(line.split("|")[2].split()[0])
    return None


def config(args, n):
    r = ph.RECIPES[args.workload]
    return {"workload": f"{args.workload}: {'x'.join(map(str, r['dims']))} @{r['spacing'][0]} mm, "
                        f"pe_dim {r['pe_dim']}, OT init + blur + {GN_ITERS[args.workload]} GN-PCG "
                        f"iterations (<=10 PCG, <=10 Armijo trials)",
            "dims": list(r["dims"]), "pe_dim": r["pe_dim"], "alpha": ALPHA, "beta": BETA,
            "gn_iters": GN_ITERS[args.workload], "pcg_max_iters": 10,
            "precond": "column" if args.precond else "jacobi",
            "pairs_per_rank_per_step": 1, "n_ranks": n,
            "l2": "value: flushed before every timed step (256 MiB write, then 256 MiB read of "
                  "another buffer: L2 left clean), outside the timed events; e2e: no flush, two "
                  "alternating slots whose per-step working sets (~140 MB each) exceed L2"}


# ------------------------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline leg)
# ------------------------------------------------------------------------------------------

def host_cores():
    """(threads the oracle may use, CPU model): the cores this process is allowed to run on."""
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return n, model


def oracle_problem(pr, threads):
    import oracle
    oracle.set_threads(threads)
    return oracle.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)


def oracle_ot(P, pr):
    """The solve's start: OT initialisation + blur and the feasible-start rule (timed)."""
    t0 = time.perf_counter()
    b, _, _ = P.solve(pr.Ip, pr.Im, gn_iters=0, init=True)
    return b, time.perf_counter() - t0


def oracle_gn(P, pr, b):
    """One Gauss-Newton iteration of the oracle's solve from b (timed): (new b, seconds)."""
    t0 = time.perf_counter()
    b, _, _ = P.solve(pr.Ip, pr.Im, b=b, gn_iters=1, init=False)
    return b, time.perf_counter() - t0


def cpu_baseline(pr, args):
    """The oracle (FP64 C, OpenMP over columns) timed on this host: one whole solve of the pair
    (OT + blur + GN_ITERS Gauss-Newton iterations) on every allowed core, and OT + one GN
    iteration on one thread (its per-pair figure extrapolated, stated as such)."""
    cores, model = host_cores()
    gn = GN_ITERS[args.workload]
    P = oracle_problem(pr, cores)
    b, t_ot = oracle_ot(P, pr)
    t_gn = []
    for _ in range(gn):
        b, t = oracle_gn(P, pr, b)
        t_gn.append(t)
    per_pair = t_ot + sum(t_gn)
    P1 = oracle_problem(pr, 1)
    b1, t1_ot = oracle_ot(P1, pr)
    _, t1_gn = oracle_gn(P1, pr, b1)
    one = t1_ot + gn * t1_gn
    return {"value": 1.0 / per_pair, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": model,
            "sample": f"one whole {args.workload} solve on {cores} threads: OT + blur "
                      f"{t_ot:.2f} s, {gn} GN iterations {sum(t_gn):.2f} s "
                      f"({min(t_gn):.2f}-{max(t_gn):.2f} s each); FP64 C oracle, OpenMP over "
                      f"columns with fixed-order sums",
            "one_thread": {"value": 1.0 / one, "unit": UNIT, "cores": 1,
                           "sample": f"OT + blur {t1_ot:.2f} s and GN iteration 1 {t1_gn:.2f} s "
                                     f"timed on one thread, extrapolated to OT + {gn} GN"}}


# ------------------------------------------------------------------------------------------
# multi-rank host logic (replicas: every rank solves its own pairs, no data-path collective)
# ------------------------------------------------------------------------------------------

def rank_env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(workload, rank):
    """Seed of the pair a rank solves: each rank gets its own problem."""
    return ph.RECIPES[workload]["seed"] + 17 * rank


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself when not distributed)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def run_reference(args):
    """The oracle as the reference arm: every step is one Gauss-Newton iteration of the oracle's
    own solve of the pair (b carried from step to step, all allowed cores), so K = GN_ITERS
    timed steps are exactly one whole solve; the pair rate adds the (separately timed) OT start.
    Rank 0 alone runs it."""
    world, rank, _ = rank_env()
    if rank != 0:
        return
    pr = ph.make_pair(args.workload)
    cores, model = host_cores()
    gn = GN_ITERS[args.workload]
    P = oracle_problem(pr, cores)
    b, t_ot = oracle_ot(P, pr)
    for _ in range(args.warmup):
        b, _ = oracle_gn(P, pr, b)
    times = []
    for _ in range(args.steps):
        b, t = oracle_gn(P, pr, b)
        times.append(t)
    t_gn = statistics.mean(times)
    per = t_ot + gn * t_gn
    v = 1.0 / per
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_gn * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded phantom standing in for HCP 3T data)",
            "config": config(args, 1),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu_model": model,
                             "sample": f"per step one GN iteration of the oracle's solve "
                                       f"(iterations {args.warmup + 1}..{args.warmup + args.steps}"
                                       f", b carried over, {t_gn:.2f} s mean); per pair OT + blur "
                                       f"({t_ot:.2f} s) + {gn} x the mean step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

class L2Flush:
    """Evicts L2 (126 MB on B300): writes a 256 MiB buffer, then reads another 256 MiB buffer,
    so that L2 ends up holding clean lines of the second one (nothing left to write back)."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        self.r = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def __call__(self):
        self.w.zero_()
        self.r.sum()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 9:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        load = [s for s in sm if mx and s > 0.3 * max(mx)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def solve_alg_bytes(nimg, nfld, es, gn):
    """Algorithmic bytes of one solve (OT + blur + gn GN iterations with gamma = 1 accepted, as the
    bench workload runs), images of es bytes per voxel: the OT shift and OT read both images
    (2 x 2 es per voxel) and write b (4), the blur's three passes read and write b (24 per node);
    per GN iteration the gamma = 1 trial evaluation reads both images (2 es per voxel) and b, q,
    grad (12 per node) and writes grad, d, e, 1/diag (16), the persistent PCG moves 400 per node
    (init + 10 iterations at 40 per iteration, the hot-path byte count for H v and the fused
    vector updates), and the update reads b, q and writes b (12)."""
    ot = 4 * es * nimg + 4 * nfld + 24 * nfld
    per_it = 2 * es * nimg + 28 * nfld + 400 * nfld + 12 * nfld
    return ot + gn * per_it


def precision_sweep(args, dev, stream, flush, n_pairs=64, reps=2):
    """The precision sweep at scale: the first n_pairs pairs of the 3T sweep (each its own images,
    together far larger than L2) solved as one batch (hysco_batch_*, schedule tuned once on f32)
    with the images stored in f32, bf16 and f16 (field, interpolation and sums single precision).
    Aggregate pairs/s and algorithmic GB/s per storage type, device-resident and end to end (the
    images uploaded from pinned host memory in the storage type and the fields downloaded, the
    copies inside the timed region), and the largest relative field difference of each
    reduced-precision solve from the f32 solve of the same pair.  The error against the double-
    precision oracle is checked by the precision test."""
    import torch

    from paper_2403_10706_b300.hysco import Hysco, HyscoBatch
    gn = GN_ITERS["3t"]
    pairs = [ph.make_sweep_pair(i) for i in range(n_pairs)]
    nimg = int(np.prod(pairs[0].dims))
    out, ref, sched = {}, None, None
    for key, td in (("f32", torch.float32), ("bf16", torch.bfloat16), ("f16", torch.float16)):
        hs = [Hysco(p.dims, p.spacing, p.pe_dim, ALPHA, BETA, dtype=td, device=dev) for p in pairs]
        nfld = int(np.prod(hs[0].field_dims))
        Ips = [torch.from_numpy(p.Ip).to(dev).to(td) for p in pairs]
        Ims = [torch.from_numpy(p.Im).to(dev).to(td) for p in pairs]
        hIp = [t.cpu().pin_memory() for t in Ips]
        hIm = [t.cpu().pin_memory() for t in Ims]
        bs = [h._new_fld() for h in hs]
        hb = [torch.empty(h.field_dims, dtype=torch.float32).pin_memory() for h in hs]
        batch = HyscoBatch(hs)
        if sched is None:
            sched = batch.tune(Ips, Ims, gn_iters=gn)
        else:
            batch.set_schedule(sched[0], sched[1])

        def solve():
            batch.solve(Ips, Ims, bs=bs, init=True, gn_iters=gn, stats=False)

        def e2e():
            for i in range(n_pairs):
                Ips[i].copy_(hIp[i], non_blocking=True)
                Ims[i].copy_(hIm[i], non_blocking=True)
            solve()
            for i in range(n_pairs):
                hb[i].copy_(bs[i], non_blocking=True)

        res = {}
        for name, fn in (("dev", solve), ("e2e", e2e)):
            fn()
            torch.cuda.synchronize()
            evs = []
            for _ in range(reps):
                flush()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            res[name] = sum(a.elapsed_time(b) for a, b in evs) / 1e3 / reps
        es = Ips[0].element_size()
        alg = n_pairs * solve_alg_bytes(nimg, nfld, es, gn)
        fields = [b.cpu().numpy() for b in bs]
        entry = {"value": n_pairs / res["dev"], "e2e": n_pairs / res["e2e"],
                 "alg_gbs": alg / res["dev"] / 1e9, "alg_bytes_per_pair": alg // n_pairs,
                 "h2d_bytes_per_pair": int(2 * nimg * es),
                 "status_nonzero": sum(1 for h in hs if h.last_status() != 0)}
        if ref is None:
            ref = fields
        else:
            entry["field_rel_diff_vs_f32"] = max(
                float(np.linalg.norm(f - r) / np.linalg.norm(r)) for f, r in zip(fields, ref))
        out[key] = entry
        del batch, hs, Ips, Ims, hIp, hIm, bs, hb
        torch.cuda.empty_cache()
    out["unit"] = UNIT
    out["gain_bf16_vs_f32"] = out["bf16"]["value"] / out["f32"]["value"]
    out["gain_f16_vs_f32"] = out["f16"]["value"] / out["f32"]["value"]
    out["e2e_gain_bf16_vs_f32"] = out["bf16"]["e2e"] / out["f32"]["e2e"]
    out["schedule"] = {"branches": sched[0], "policy": sched[1]}
    out["sample"] = (f"sweep pairs 0..{n_pairs - 1} of 288 (3T shape, shared field map, contrast "
                     f"U(0.2, 1), N(0, 0.03) noise; images {n_pairs * 2 * nimg * 4 / 1e9:.2f} GB "
                     f"in f32), one batched solve of all of them per timed step, {reps} steps, L2 "
                     f"flushed per step")
    return out


def batch_bench(dev, stream, flush, reps=2):
    """The uneven batch: 64 pairs (22 of the 3T shape, 21 7T-shaped, 21 of 96x96x60, PE along
    axis 0 or 1, field-map peaks U(4, 10) voxels), OT init + 20 GN-PCG iterations each, solved
    by one autotuned batched solve (hysco_batch_*) and by 64 sequential plain solves
    (hysco_solve, each its own cached graph); L2 flushed before each timed run."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import torch

    from paper_2403_10706_b300.hysco import Hysco, HyscoBatch
    recipes = ph.batch_recipes()
    workers = max(1, min(16, len(os.sched_getaffinity(0))))
    t0 = time.time()
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        pairs = list(ex.map(ph.make_pair, recipes))
    gen_s = time.time() - t0
    gn = GN_ITERS["3t"]
    hs = [Hysco(p.dims, p.spacing, p.pe_dim, ALPHA, BETA, device=dev) for p in pairs]
    Ips = [torch.from_numpy(p.Ip).to(dev) for p in pairs]
    Ims = [torch.from_numpy(p.Im).to(dev) for p in pairs]
    bs = [h._new_fld() for h in hs]
    batch = HyscoBatch(hs)
    t0 = time.time()
    sched = batch.tune(Ips, Ims, gn_iters=gn)
    tune_s = time.time() - t0

    def run_batch():
        batch.solve(Ips, Ims, bs=bs, init=True, gn_iters=gn, stats=False)

    def run_seq():
        for i, h in enumerate(hs):
            h.solve(Ips[i], Ims[i], b=bs[i], gn_iters=gn, init=True, stats=False)

    out = {}
    for name, fn in (("batched", run_batch), ("sequential", run_seq)):
        fn()
        torch.cuda.synchronize()
        evs = []
        for _ in range(reps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        t = sum(a.elapsed_time(b) for a, b in evs) / 1e3
        out[name] = len(pairs) * reps / t
        out[name + "_status_nonzero"] = sum(1 for h in hs if h.last_status() != 0)
    # two fixed schedules beside the tuned one: waves whose PCGs share a launch per GN step
    # (policy 4) and waves whose whole GN loops are one persistent launch (policy 7)
    fixed = {}
    for label, pol in (("pcg_waves_policy4", 4), ("gn_loop_waves_policy7", 7)):
        try:
            batch.set_schedule(2, pol)
        except RuntimeError:
            continue
        run_batch()
        torch.cuda.synchronize()
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_batch()
        e1.record(stream)
        torch.cuda.synchronize()
        fixed[label] = len(pairs) / (e0.elapsed_time(e1) / 1e3)
    batch.set_schedule(sched[0], sched[1])
    out.update({"unit": UNIT, "speedup": out["batched"] / out["sequential"],
                "fixed_schedules_2_branches": fixed,
                "schedule": {"branches": sched[0], "block_share_policy": sched[1],
                             "pcg_grid_blocks": sched[2]},
                "tune_s": tune_s, "generate_s": gen_s,
                "workload": "64 pairs: 22x 144x168x111, 21x 130x130x85, 21x 96x96x60 (seeded "
                            "shuffle), PE axis 0 or 1, field peaks U(4, 10) voxels; OT + 20 GN "
                            "each", "reps": reps})
    del batch
    return out


def run_ours(args):
    import torch

    from paper_2403_10706_b300 import _lib
    from paper_2403_10706_b300 import build as b
    from paper_2403_10706_b300.hysco import Hysco

    b.build()
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    pr = ph.make_pair(args.workload, seed=rank_seed(args.workload, rank))
    gn = GN_ITERS[args.workload]
    h = Hysco(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA, device=dev)
    Ip = torch.from_numpy(pr.Ip).to(dev)
    Im = torch.from_numpy(pr.Im).to(dev)
    b_out = torch.empty(h.field_dims, dtype=torch.float32, device=dev)
    flush = L2Flush(dev)

    def step():
        h.solve(Ip, Im, b=b_out, gn_iters=gn, init=True, precond=args.precond, stats=False,
                pcg_path=args.pcg_path)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    status = h.last_status()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local).__enter__()
    for s0, s1 in evs:
        flush()
        s0.record(stream)
        step()
        s1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = [s0.elapsed_time(s1) for s0, s1 in evs]
    total_s = max_over_ranks(sum(ms) / 1e3, dist, dev)
    value = job_throughput(world, args.steps, total_s)

    # end to end through the public API, as a serving loop runs it: every step uploads its pair's
    # images from pinned host memory and downloads the solved field, on a copy stream.  Two
    # handle/buffer slots alternate, so step i+1's upload overlaps step i's solve and step i's
    # download overlaps step i+1's solve; one event pair brackets all steps.  No explicit L2
    # flush here: a slot's solve touches ~140 MB (images, field, nine solver arrays), so with two
    # alternating slots each step's working set exceeds the 126 MB L2 left by the step before.
    copy = torch.cuda.Stream(dev)
    h2 = Hysco(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA, device=dev)
    slots = [(h, Ip, Im, b_out),
             (h2, torch.empty_like(Ip), torch.empty_like(Im), torch.empty_like(b_out))]
    hIp = torch.from_numpy(pr.Ip).pin_memory()
    hIm = torch.from_numpy(pr.Im).pin_memory()
    hbs = [torch.empty(h.field_dims, dtype=torch.float32).pin_memory() for _ in slots]
    for hh, a, c, bb in slots:   # warm-up: capture each slot's graph
        a.copy_(hIp)
        c.copy_(hIm)
        hh.solve(a, c, b=bb, gn_iters=gn, init=True, precond=args.precond, stats=False,
                 pcg_path=args.pcg_path)
    torch.cuda.synchronize()
    n_e2e = max(4, args.steps)
    up = [torch.cuda.Event() for _ in slots]
    done = [torch.cuda.Event() for _ in slots]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(copy)
    with torch.cuda.stream(copy):
        slots[0][1].copy_(hIp, non_blocking=True)
        slots[0][2].copy_(hIm, non_blocking=True)
    up[0].record(copy)
    for i in range(n_e2e):
        k = i % 2
        hh, a, c, bb = slots[k]
        stream.wait_event(up[k])
        hh.solve(a, c, b=bb, gn_iters=gn, init=True, precond=args.precond, stats=False,
                 pcg_path=args.pcg_path)
        done[k].record(stream)
        if i + 1 < n_e2e:   # upload the next step's images into the other slot once it is free
            nk = 1 - k
            if i >= 1:
                copy.wait_event(done[nk])
            with torch.cuda.stream(copy):
                slots[nk][1].copy_(hIp, non_blocking=True)
                slots[nk][2].copy_(hIm, non_blocking=True)
            up[nk].record(copy)
        copy.wait_event(done[k])
        with torch.cuda.stream(copy):
            hbs[k].copy_(bb, non_blocking=True)
    e1.record(copy)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
    e2e = {"value": job_throughput(world, n_e2e, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(Ip.numel() * 4 + Im.numel() * 4),
           "d2h_bytes_per_step": int(b_out.numel() * 4),
           "steps": n_e2e, "pipeline": "double-buffered: step i+1's upload and step i's download "
                                       "overlap the solves on a copy stream",
           "l2": "no explicit flush: two alternating handle/buffer slots, each solve touching "
                 "~140 MB, so every step's working set exceeds the 126 MB L2"}
    del h2, slots

    # Roofline of the dominant kernel, the persistent Jacobi-PCG kernel (one launch per GN step),
    # timed alone through hysco_pcg on this stream with L2 flushed before each launch.  rtol = 0
    # makes every launch run exactly 10 iterations.  Algorithmic bytes per field node (4-byte
    # floats) with r, p, Hp of every group on chip (shared memory for the whole launch): init
    # reads grad, 1/diag and writes x, z (16); iteration 0 reads z, d, e (12), then reads 1/diag
    # and writes x, z (12); every later iteration reads z, d, e (12), then reads 1/diag, x and
    # writes x, z (16).  Groups whose r, p, Hp stay in global memory add, per node, the write of
    # r at init (4), of p, Hp at iteration 0 (8) and the reads of p, Hp, r and write of r in
    # every phase B (16), and the read and write of p, Hp in every later phase A (16).
    nimg = int(np.prod(pr.dims))
    nfld = int(np.prod(h.field_dims))
    peak, peak_src = peaks()
    terms = torch.empty(4, dtype=torch.float64, device=dev)
    g = torch.empty_like(b_out)
    q = torch.empty_like(b_out)
    h.eval(Ip, Im, b_out, grad=g, terms=terms)
    rhs = -g

    def time_launches(fn, n=20):
        for _ in range(3):
            fn()
        evs = []
        for _ in range(n):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)

    # The one-barrier form (--pcg-path 3) moves per node: phase 0 reads grad, 1/diag, d, e and
    # writes r, w (24); phase 1 reads r, w, 1/diag, d, e and writes x, p, q, r, w (40); phases
    # 2..9 read r, w, q, 1/diag, p, x, d, e and write x, p, q, r, w (52); the last phase skips
    # the stencil: reads r, w, q, 1/diag, p, x and writes x, p, q, r (40).
    pcg_iters = 10
    fused = args.pcg_path == 3
    grid, onchip, slots, pblock = h.pcg_plan()
    fe = h.field_dims
    n4 = fe[0] * fe[1] * ((fe[2] + 3) // 4)
    f_on = min(n4, onchip * grid * pblock) / n4 if grid else 0.0    # share of groups on chip
    if fused:
        pcg_bytes = nfld * (24 + 40 + (pcg_iters - 2) * 52 + 40)
    elif args.pcg_path == 1:
        pcg_bytes = nfld * (20 + 20 + 28 + (pcg_iters - 1) * (28 + 32))
    else:
        off = 1.0 - f_on
        pcg_bytes = int(nfld * (16 + 4 * off + 12 + 8 * off + 12 + 16 * off +
                                (pcg_iters - 1) * (12 + 16 * off + 16 + 16 * off)))
    pcg_ms = time_launches(lambda: h.pcg(rhs, max_iters=pcg_iters, rtol=0.0, out=q,
                                         pcg_path=args.pcg_path))
    achieved = pcg_bytes / (pcg_ms / 1e3) / 1e9
    kname = {1: "k_hv + k_pcg_update_jacobi (separate)", 3: "k_pcg_fused<jacobi>"}.get(
        args.pcg_path, "k_pcg_persistent<jacobi>")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": recorded_traffic("k_pcg_persistent_3t.md", PCG_SOURCES)
            if args.workload == "3t" and args.pcg_path in (0, 2) else None,
            "kernel": kname,
            "peak_source": peak_src, "alg_bytes_per_launch": pcg_bytes, "launch_ms": pcg_ms,
            "pcg_plan": {"grid": grid, "block": pblock, "onchip_slots": onchip,
                         "slots": slots, "onchip_share": f_on},
            "note": "10 PCG iterations per launch; r, p, Hp of the on-chip share stay in shared "
                    "memory; z, x, d, e, 1/diag (54 MB) are largely L2-resident within a launch, "
                    "so achieved algorithmic bandwidth may exceed the HBM copy peak"}
    # the eval kernel (J, grad J, GN coefficients): read I+, I- (4 B each per voxel) and b
    # (4 B per node); write grad, d, e, 1/diag (4 B each per node)
    alg_eval = 8 * nimg + 20 * nfld
    eval_ms = time_launches(lambda: h.eval(Ip, Im, b_out, grad=g, terms=terms))
    ach_eval = alg_eval / (eval_ms / 1e3) / 1e9
    # the corrected-image adjoint (backward of hysco_correct): reads I+, I-, g+, g- (16 B per
    # voxel) and b (4 B per node, once per image pass and once for the field pass), writes dI+,
    # dI- (8 B per voxel) and db (4 B per node)
    gT = torch.randn(pr.dims, device=dev, dtype=torch.float32)
    dIp, dIm, dbb = (torch.empty_like(gT), torch.empty_like(gT), torch.empty_like(b_out))
    alg_adj = 24 * nimg + 16 * nfld
    adj_ms = time_launches(lambda: h.lib.hysco_correct_adjoint(
        h._h, h._img(Ip, "Ip"), h._img(Im, "Im"), h._fld(b_out, "b"), h._img_f32(gT, "gTp"),
        h._img_f32(gT, "gTm"), h._img_f32(dIp, "dIp"), h._img_f32(dIm, "dIm"),
        h._fld(dbb, "db"), stream.cuda_stream))
    adjoint = {"launch_ms": adj_ms, "alg_bytes_per_launch": alg_adj,
               "achieved": alg_adj / (adj_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
               "frac": alg_adj / (adj_ms / 1e3) / 1e9 / peak,
               "kernel": "k_image_adjoint x2 + k_field_adjoint"}
    # the least-squares correction (a per-column banded solve): reads I+, I- (8 B per voxel) and
    # b (4 B per node), writes the image (4 B per voxel); its scratch traffic (band assembly and
    # factorisation) stays per column in L1 / L2
    lsout = torch.empty(pr.dims, dtype=torch.float32, device=dev)
    nbad = torch.zeros(1, dtype=torch.int32, device=dev)
    alg_ls = 12 * nimg + 4 * nfld
    ls_ms = time_launches(lambda: h.lib.hysco_ls_correct(
        h._h, h._img(Ip, "Ip"), h._img(Im, "Im"), h._fld(b_out, "b"), 1e-6,
        lsout.data_ptr(), nbad.data_ptr(), stream.cuda_stream))
    ls = {"launch_ms": ls_ms, "alg_bytes_per_launch": alg_ls,
          "achieved": alg_ls / (ls_ms / 1e3) / 1e9, "unit": "GB/s", "kernel": "k_ls_correct",
          "columns_skipped": int(nbad.item())}
    # the other hot-path entry points, each timed alone (L2 flushed before every call) with its
    # minimal algorithmic bytes per node (4-byte floats; images 4 B per voxel and image):
    #   hysco_init_ot   read I+, I- (8 per voxel), write b (4 per node)         [shift, OT, blur]
    #   hysco_hessvec   read v, d, e (12), write Hv (4)                        [one stencil kernel]
    #   hysco_precond   read r, d, e (12), write z (4): per-column tridiagonal factor and solve
    def table_row(ms, alg, launches):
        return {"launch_ms": ms, "alg_bytes_per_call": alg, "launches": launches,
                "achieved": alg / (ms / 1e3) / 1e9, "unit": "GB/s", "frac": alg / (ms / 1e3) / 1e9 / peak}
    bt = torch.empty_like(b_out)
    vv = torch.randn_like(b_out)
    hv_out, pc_out = torch.empty_like(b_out), torch.empty_like(b_out)
    kernels = {
        "hysco_init_ot": table_row(time_launches(lambda: h.init_ot(Ip, Im, out=bt)),
                                   8 * nimg + 4 * nfld, "k_ot_shift, k_ot, k_blur3"),
    }
    h.eval(Ip, Im, b_out, grad=g, terms=terms)   # the linearisation the next two calls use
    kernels["hysco_hessvec"] = table_row(time_launches(lambda: h.hessvec(vv, out=hv_out)),
                                         16 * nfld, "k_hv_caller")
    kernels["hysco_precond_column"] = table_row(
        time_launches(lambda: h.precond(vv, kind=_lib.PC_COLUMN, out=pc_out)), 16 * nfld,
        "k_col_factor, k_col_solve")
    # the paper's 7T acquisition size (200 x 200 x 132, PE axis 0): a field of 5.3 M nodes, twice
    # what the persistent PCG keeps on chip, so half its slots keep r, p, Hp in global memory
    extra = None
    if args.workload == "3t" and not args.no_extra_shapes:
        px = ph.make_pair("7t_paper")
        hx = Hysco(px.dims, px.spacing, px.pe_dim, ALPHA, BETA, device=dev)
        Ipx, Imx = torch.from_numpy(px.Ip).to(dev), torch.from_numpy(px.Im).to(dev)
        bx = hx._new_fld()
        x_ms = time_launches(lambda: hx.solve(Ipx, Imx, b=bx, gn_iters=20, init=True,
                                              stats=False), n=5)
        gridx, onx, slotsx, _ = hx.pcg_plan()
        extra = {"7t_paper": {"dims": list(px.dims), "pe_dim": px.pe_dim, "gn_iters": 20,
                              "ms_per_solve": x_ms, "pairs_per_s": 1e3 / x_ms,
                              "status": hx.last_status(),
                              "pcg_onchip_slots": [onx, slotsx]}}
        del hx, Ipx, Imx, bx
    # ADMM (Sec. 2.3.2) on the same pair: OT + 20 iterations of 2 GN steps (BlockPCG directions)
    # each, against the GN solve's 20 iterations; the z-update's four per-plane products move
    # 2 * E * nB * nA * (nB + nA) flops each way (forward and inverse transform)
    ab = torch.empty_like(b_out)
    admm_ms = None
    if not args.no_admm:
        admm_ms = time_launches(lambda: h.admm(Ip, Im, b=ab, init=1, admm_iters=20, tol=0.0,
                                               stats=False), n=5)
        _, ast = h.admm(Ip, Im, b=ab, init=1, admm_iters=20, tol=0.0)
        # the z-update alone (hysco_admm_zsolve) on both arithmetic paths
        zv = torch.randn(h.field_dims, device=dev, generator=torch.Generator(device=dev).manual_seed(7))
        zo = torch.empty_like(zv)
        z_path = h.zsolve_path()
        z_ms = {}
        for zp in ((0, 1) if z_path == 0 else (1,)):
            h.set_zsolve_path(zp)
            z_ms[zp] = time_launches(lambda: h.admm_zsolve(zv, 40.0, out=zo), n=20)
        h.set_zsolve_path(z_path)
    _, gst = h.solve(Ip, Im, gn_iters=gn)
    fe = h.field_dims
    plane = [fe[a] for a in range(3) if a != pr.pe_dim]
    zflop = 2 * 2 * fe[pr.pe_dim] * plane[0] * plane[1] * (plane[0] + plane[1])
    # the work the timed solves do (deterministic: the same trajectory as this solve's)
    gs = gst.cpu().numpy()
    work = {"gn_iters": int(gn), "pcg_iterations": int(np.nansum(gs[:, 7])),
            "ls_trials": int(np.nansum(gs[:, 9])),
            "gamma_1_accepted": int(np.sum(gs[:, 6] == 1.0)),
            "J_at_first_gn_iter": float(gs[0, 0]), "J_at_last_gn_iter": float(gs[-1, 0])}
    admm = None
    if admm_ms is not None:
        admm = {"iters": 20, "gn_steps_per_b_update": 2, "ms_per_run": admm_ms,
                "pairs_per_s": 1e3 / admm_ms, "J_final": float(ast[-1, 0].item()),
                "J_gn_solve": float(gst[-1, 0].item()), "rho_final": float(ast[-1, 2].item()),
                "z_update_flop_per_iter": zflop, "status": h.last_status(),
                "note": "L2 flushed before each run; J at the last iterate of each optimiser"}
        tfp, tfsrc = tf32_peak()
        zu = {"path": "tensor cores (tcgen05 kind::tf32, TF32 split in shared memory)" if z_path == 0
              else "CUDA cores (FP32)",
              "ms": z_ms[z_path], "ms_cuda_cores": z_ms[1],
              "speedup_vs_cuda_cores": z_ms[1] / z_ms[z_path],
              "note": "hysco_admm_zsolve at 3T (the rhs split, four products, copy out of the "
                      "pitched field), L2 flushed before each call"}
        if z_path == 0:
            # three TF32 products per basis product (hi hi, hi lo, lo hi)
            zu["tensor_roofline"] = {"bound": "tensor", "achieved": 3 * zflop / (z_ms[0] / 1e3) / 1e12,
                                     "peak": tfp, "unit": "TFLOP/s",
                                     "frac": 3 * zflop / (z_ms[0] / 1e3) / 1e12 / tfp,
                                     "peak_source": tfsrc,
                                     "flop_per_call": 3 * zflop}
        admm["z_update"] = zu
    eval_roof = {"bound": "hbm", "achieved": ach_eval, "peak": peak, "unit": "GB/s",
                 "frac": ach_eval / peak,
                 "traffic": recorded_traffic("k_eval_3t.md", EVAL_SOURCES)
                 if args.workload == "3t" else None,
                 "kernel": "k_eval<float>",
                 "alg_bytes_per_launch": alg_eval, "launch_ms": eval_ms}
    clk.__exit__(None, None, None)   # sampled over the timed solves, e2e and roofline launches
    # the eval kernel is bound by instruction issue: warp instructions per launch (ncu) over the
    # issue capacity in the measured launch time (4 schedulers per SM, one instruction per cycle,
    # at the SM clock sampled during the run)
    winst = recorded_warp_instructions("k_eval_3t.md", EVAL_SOURCES) \
        if args.workload == "3t" else None
    clk_mhz = clk.summary().get("sm_mhz") or 2032.0
    if winst is not None:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        cap = sms * 4 * clk_mhz * 1e6 * eval_ms / 1e3
        eval_roof["issue"] = {"warp_instructions_per_launch": winst, "issue_capacity": cap,
                              "frac": winst / cap, "sm_mhz": clk_mhz}

    prec = None
    if rank == 0 and args.workload == "3t" and not args.no_precision:
        prec = precision_sweep(args, dev, stream, flush)
    batch = None
    if rank == 0 and args.workload == "3t" and not args.no_batch:
        batch = batch_bench(dev, stream, flush)

    if rank == 0:
        # OT: shift, OT, blur, then the feasible-start check and scale; per GN step: eval (a
        # no-op when the previous gamma = 1 trial was accepted), PCG (1 persistent launch, or
        # init + 2 per iteration), the gamma = 1 trial evaluation, one launch for the remaining
        # halvings (a no-op when gamma = 1 is accepted), update.  Kernels replayed from the CUDA
        # graph count as launches.
        persistent = args.precond == 0 and args.pcg_path != 1   # 0, 2 and 3 are one launch
        pcg_launches = 1 if persistent else 1 + 2 * 10 + (1 if args.precond else 0)
        launches_per_step = 5 + gn * (1 + pcg_launches + 2 + 1)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded phantom standing in for HCP 3T data)",
                "config": config(args, world), "status": status,
                "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "roofline": roof, "eval_roofline": eval_roof, "adjoint": adjoint,
                "ls_correct": ls, "admm": admm, "kernel_table": kernels, "work": work,
                "extra_shapes": extra}
        if prec is not None:
            line["precision"] = prec
        if batch is not None:
            line["batch"] = batch
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(pr, args)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
