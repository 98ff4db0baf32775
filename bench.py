"""Throughput benchmark: corrected 3T-shaped volume pairs per second at a fixed GN iteration count.

One step = one full solve of one 144x168x111 (1.25 mm, PE along the 168 axis) synthetic pair:
OT initialisation with blur + 20 Gauss-Newton iterations, each with up to 10 Jacobi-PCG
iterations and an Armijo line search (the paper's default method, Sec. 2.2-2.3.1), inputs
resident in HBM.  L2 is flushed (a 256 MiB write) before every timed step; each step is timed
with CUDA events on the launching stream and the flush is outside the events.

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
GN_ITERS = {"3t": 20, "7t": 20, "small": 20, "tiny": 10}
ALPHA, BETA = 300.0, 1e4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3t", choices=list(GN_ITERS))
    ap.add_argument("--precond", type=int, default=0)
    ap.add_argument("--pcg-path", type=int, default=0,
                    help="0 auto (persistent PCG kernel when possible), 1 separate kernels")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def config(args, n):
    r = ph.RECIPES[args.workload]
    return {"workload": f"{args.workload}: {'x'.join(map(str, r['dims']))} @{r['spacing'][0]} mm, "
                        f"pe_dim {r['pe_dim']}, OT init + blur + {GN_ITERS[args.workload]} GN-PCG "
                        f"iterations (<=10 PCG, <=10 Armijo trials)",
            "dims": list(r["dims"]), "pe_dim": r["pe_dim"], "alpha": ALPHA, "beta": BETA,
            "gn_iters": GN_ITERS[args.workload], "pcg_max_iters": 10,
            "precond": "column" if args.precond else "jacobi",
            "pairs_per_rank_per_step": 1, "n_ranks": n,
            "l2": "flushed (256 MiB write) before every timed step, outside the timed events"}


# ------------------------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline leg)
# ------------------------------------------------------------------------------------------

def oracle_sample(pr, gn_sample=2):
    """Times the oracle on a bounded sample of one solve: the OT initialisation plus `gn_sample`
    GN iterations, extrapolated to the full fixed iteration count."""
    import oracle
    P = oracle.Problem(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA)
    t0 = time.perf_counter()
    b0 = P.ot_init(pr.Ip, pr.Im, 1e-3, contract=False, blur=True)
    t_ot = time.perf_counter() - t0
    t0 = time.perf_counter()
    P.solve(pr.Ip, pr.Im, b=b0, gn_iters=gn_sample, init=False)
    t_gn = (time.perf_counter() - t0) / gn_sample
    return t_ot, t_gn


def cpu_baseline(pr, args):
    t_ot, t_gn = oracle_sample(pr)
    per_pair = t_ot + GN_ITERS[args.workload] * t_gn
    return {"value": 1.0 / per_pair, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one {args.workload} pair: OT init + 2 GN iterations timed "
                      f"(OT {t_ot:.2f} s, {t_gn:.2f} s per GN iteration), extrapolated to "
                      f"OT + {GN_ITERS[args.workload]} GN; single-threaded FP64 C oracle"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pr = ph.make_pair(args.workload)
    for _ in range(args.warmup):
        oracle_sample(pr, gn_sample=1)
    times = []
    for _ in range(args.steps):
        t_ot, t_gn = oracle_sample(pr, gn_sample=1)
        times.append(t_ot + GN_ITERS[args.workload] * t_gn)
    per = statistics.mean(times)
    v = 1.0 / per
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded phantom standing in for HCP 3T data)",
            "config": config(args, 1),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "per step: OT init + 1 GN iteration of one pair, "
                                       "extrapolated to the full iteration count"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

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
                 "--format=csv,noheader,nounits", "-lms", "200"],
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


def run_ours(args):
    import torch

    from paper_2403_10706_b300 import build as b
    from paper_2403_10706_b300.hysco import Hysco

    b.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    pr = ph.make_pair(args.workload, seed=ph.RECIPES[args.workload]["seed"] + 17 * rank)
    gn = GN_ITERS[args.workload]
    h = Hysco(pr.dims, pr.spacing, pr.pe_dim, ALPHA, BETA, device=dev)
    Ip = torch.from_numpy(pr.Ip).to(dev)
    Im = torch.from_numpy(pr.Im).to(dev)
    b_out = torch.empty(h.field_dims, dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2

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
    with ClockSampler(local) as clk:
        for s0, s1 in evs:
            flush.zero_()
            s0.record(stream)
            step()
            s1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = [s0.elapsed_time(s1) for s0, s1 in evs]
    total_s = sum(ms) / 1e3
    if dist:
        t = torch.tensor([total_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * args.steps / total_s

    # end to end through the public API: pinned host images in, field out, every step
    hIp = torch.from_numpy(pr.Ip).pin_memory()
    hIm = torch.from_numpy(pr.Im).pin_memory()
    hb = torch.empty(h.field_dims, dtype=torch.float32).pin_memory()
    e2e_ms = []
    for i in range(max(3, args.steps // 2)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Ip.copy_(hIp, non_blocking=True)
        Im.copy_(hIm, non_blocking=True)
        step()
        hb.copy_(b_out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_s = sum(e2e_ms) / 1e3
    if dist:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * len(e2e_ms) / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(Ip.numel() * 4 + Im.numel() * 4),
           "d2h_bytes_per_step": int(b_out.numel() * 4)}

    # roofline of the eval kernel (J, grad J and GN coefficients), timed alone on this stream:
    # algorithmic bytes per launch = read I+, I- (4 B each per cell) and b (4 B per node), write
    # grad, d, e (4 B each per node)
    nimg = int(np.prod(pr.dims))
    nfld = int(np.prod(h.field_dims))
    alg_bytes = 8 * nimg + 16 * nfld
    terms = torch.empty(4, dtype=torch.float64, device=dev)
    g = torch.empty_like(b_out)
    for _ in range(3):
        h.eval(Ip, Im, b_out, grad=g, terms=terms)
    kev = []
    for _ in range(20):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.eval(Ip, Im, b_out, grad=g, terms=terms)
        e1.record(stream)
        kev.append((e0, e1))
    torch.cuda.synchronize()
    k_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in kev)
    peak, peak_src = peaks()
    achieved = alg_bytes / (k_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "kernel": "k_eval<float>",
            "peak_source": peak_src, "alg_bytes_per_launch": alg_bytes,
            "launch_ms": k_ms}

    if rank == 0:
        launches_per_step = 3 + gn * (1 + 1 + 2 * 10 + 3 + 1) + (gn if args.precond else 0)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_s * 1e3 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded phantom standing in for HCP 3T data)",
                "config": config(args, world), "status": status,
                "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "roofline": roof}
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
