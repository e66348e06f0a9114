"""Benchmark: PDHG vector-OMT solves on the 256 x 256, k = 3 colour-image workload.

One step = solving the workload once for each alpha in {0.1, 1, 10} from the
zero iterate until relative gap and relative residual are both <= 1e-5, with a
cap of 50,000 iterations (Section 7.2 iteration, complete channel graph K3,
||u||_{1,2}, ||w||_1, the paper's step-size rule with tau = 3).  The metric is
grid-point iterations per second summed over the whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle (the
reference implementation of this repository) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, K, ALPHAS, TOL, CAP = 256, 3, (0.1, 1.0, 10.0), 1e-5, 50000
CHECK_EVERY = 100
EDGES = [(0, 1), (0, 2), (1, 2)]
BYTES_PER_GP_IT = 4 * (7 * K + 2 * len(EDGES))   # read phi,u_x,u_y,w,b; write phi,u_x,u_y,w (FP32)
WORKLOAD = ("vector OMT, 256x256 grid, k=3 colour-image densities (seed 1002), complete graph K3, "
            "alpha in {0.1,1,10}, ||u||_{1,2} ||w||_1, tau=3, to rel gap and rel res <= 1e-5, cap 50000 it")
METRIC = "PDHG grid-point-iterations/s"
UNIT = "grid-point-iterations/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic_record():
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        rec = dict(line.strip().split("=", 1) for line in open(path) if "=" in line and not line.startswith("#"))
    except OSError:
        return None
    src = os.path.join(ROOT, "paper_1712_10279_gb300", "csrc", rec.get("source", ""))
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if digest != rec.get("sha256_16"):
        return None
    return rec


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _cpu_cores():
    return os.cpu_count() or 1


def oracle_sample(seconds_target=12.0):
    """Time the FP64 oracle (one thread) on a bounded sample of the workload: the first T
    iterations of the alpha = 1 solve from zero."""
    import oracle
    from paper_1712_10279_gb300 import synthetic as S
    r0, r1 = S.color_image_pair(N, K, seed=1002)
    r0 = r0.astype(np.float32).astype(np.float64)
    r1 = r1.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    oracle.vomt_solve(r0, r1, EDGES, 1.0, max_iters=5, check_every=5)
    per = (time.perf_counter() - t0) / 5
    T = int(max(10, min(3000, seconds_target / max(per, 1e-6))))
    T = (T // 10) * 10
    t0 = time.perf_counter()
    oracle.vomt_solve(r0, r1, EDGES, 1.0, max_iters=T, check_every=100)
    dt = time.perf_counter() - t0
    return {"value": N * N * T / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "first %d PDHG iterations (checks every 100) of the alpha=1 solve, 256x256 k=3, FP64, "
                      "one thread, %.1f s" % (T, dt)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = []
    samp = None
    for _ in range(args.warmup + args.steps):
        samp = oracle_sample(seconds_target=4.0)
        steps.append(samp)
    timed = steps[args.warmup:]
    v = statistics.mean(s["value"] for s in timed)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "k": K, "sample": "bounded: " + samp["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": samp["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1712_10279_gb300 as V
    from paper_1712_10279_gb300 import synthetic as S

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    r0, r1 = S.color_image_pair(N, K, seed=1002 + 1000 * rank)
    h0, h1 = r0.astype(np.float32), r1.astype(np.float32)
    d0, d1 = torch.from_numpy(h0).to(dev), torch.from_numpy(h1).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def step(results):
        for a in ALPHAS:
            sol = V.solve(d0, d1, EDGES, a, max_iters=CAP, check_every=CHECK_EVERY, tol_gap=TOL, tol_res=TOL,
                          engine=args.engine)
            results.append(sol.result)

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local_rank) if rank == 0 else None
    step_ms, results = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        step(results)
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop() if clk else None
    total_ms = sum(step_ms)
    gp_it = sum(N * N * r["iters"] for r in results)
    launches = sum(r["launches"] for r in results)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        g = torch.tensor([float(gp_it)], device=dev, dtype=torch.float64)
        dist.all_reduce(g)
        gp_it = float(g.item())
    value = gp_it / (total_ms / 1e3)

    # end to end through the host-buffer entry point: copies inside the timed region
    e2e_ms = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_iters = 0
        for a in ALPHAS:
            sol = V.solve_host(h0, h1, EDGES, a, max_iters=CAP, check_every=CHECK_EVERY, tol_gap=TOL, tol_res=TOL,
                               engine=args.engine, device=local_rank)
            e2e_iters += sol.result["iters"]
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = world * N * N * e2e_iters / (statistics.mean(e2e_ms) / 1e3)
    l = len(EDGES)
    h2d = len(ALPHAS) * 2 * K * N * N * 4
    d2h = len(ALPHAS) * (3 * K + l) * N * N * 4

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    # dominant kernel: the PDHG iteration; its algorithmic bytes over the timed GPU time
    achieved = BYTES_PER_GP_IT * (gp_it / world) / (total_ms / 1e3) / 1e9
    trec = _traffic_record()
    traffic = None
    if trec and results:
        traffic = float(trec["dram_bytes_per_iteration"]) * (sum(r["iters"] for r in results) / len(results))
    engine = results[0]["engine"] if results else args.engine
    per_alpha = {}
    for q, a in enumerate(ALPHAS):
        rs = [results[s * len(ALPHAS) + q] for s in range(args.steps)]
        per_alpha["alpha=%g" % a] = {"iters": rs[-1]["iters"], "rel_gap": rs[-1]["rel_gap"],
                                     "rel_res": rs[-1]["rel_res"], "primal": rs[-1]["primal"],
                                     "converged": rs[-1]["status"] == 0}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "k": K, "edges": l, "alphas": list(ALPHAS), "tol": TOL,
                   "cap": CAP, "check_every": CHECK_EVERY, "engine": engine,
                   "l2": "flushed (512 MB write) between timed steps",
                   "parallelism": "independent replicas, one per GPU" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_grid_point_iteration": BYTES_PER_GP_IT},
        "time_to_tolerance": per_alpha,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample()
        line["cpu_baseline"]["host_cores_available"] = _cpu_cores()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--engine", default="auto", choices=["auto", "stream", "resident"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
