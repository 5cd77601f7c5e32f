"""Benchmark: H-LU factorization seconds on one GB300 (and model GFLOP/s), plus solve latency.

A step is one hm_lu of the resident H-matrix: the task graph of the paper's semi-automatic
construction executed wave by wave in batched FP64 kernels (dense leaf LU / solves / GEMMs
and rounded truncations of every low-rank update).  Default workload: n = 131072 points
uniform on the unit-cube surface, a_ij = 1/(4 pi (|x_i - x_j| + h)), leaf 64, eta 2,
eps 1e-6, rank cap 64 (the metric's configuration); the 13 GB of block values are far
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints one JSON line; `value` is seconds per factorization (lower is better).  N > 1 (torchrun)
runs one independent replica per GPU (the H-LU of one matrix does not shard); value = the
slowest replica's seconds per step / N (factorizations of the whole job per second, inverted).
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hm_workloads as W  # noqa: E402

FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07       # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
# DRAM bytes (read + write) per counted FLOP, from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum): k_gemm, every launch of one H-LU of the n = 8192 cube (1425 launches,
# 7279.3 MB + 466.9 MB for 26.04 GFLOP; profiles/k_gemm_dram_cube8192.md); k_core, two launches of
# the n = 32768 sphere step (6 cores: 285.7 kB for 9.0379 MFLOP). A launch's traffic is taken as
# this ratio times its FLOPs.
PROFILED_BYTES_PER_FLOP = {"gemm": (7279340800.0 + 466858496.0) / 26040271168.0,
                           "core": 285696.0 / 9037896.0}
KINDS = ("getrf", "trsm", "gemm", "copy", "stack", "core", "eval", "aca")
METRIC = "H-LU factorization seconds at {w}"
WORKLOAD_TEXT = {
    "cube131072": "n=131072 uniform on the unit-cube surface, 1/(4pi(r+h)), leaf 64, eta 2, eps 1e-6, rank cap 64, FP64",
    "sphere32768": "n=32768 jittered Fibonacci sphere, 1/(4pi(r+h)), leaf 64, eta 2, eps 1e-6, rank cap 64, FP64",
    "sphere8192": "n=8192 jittered Fibonacci sphere, 1/(4pi(r+h)), leaf 64, eta 2, eps 1e-6, rank cap 64, FP64",
    "sphere2048": "n=2048 jittered Fibonacci sphere, 1/(4pi(r+h)), leaf 64, eta 2, eps 1e-4, rank cap 64, FP64",
}
ORACLE_SAMPLE = {"cube131072": ("cube", 2048, 1e-6), "sphere32768": ("sphere", 2048, 1e-6),
                 "sphere8192": ("sphere", 2048, 1e-6),
                 "sphere2048": ("sphere", 2048, 1e-4)}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        try:
            p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                  "--format=csv,noheader,nounits", "-lms", "200"],
                                 stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        self._p = p
        for line in p.stdout:
            if self._stop.is_set():
                break
            self.rows.append([x.strip() for x in line.split(",")])
        p.terminate()

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self._stop.set()
        try:
            self._p.terminate()
        except Exception:
            pass
        self._t.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(workload, repeat=3, parallel=True):
    """The FP64 oracle on the host cores, on a bounded sample of the workload (same geometry,
    seed and eps, n = 2048): the recursive H-LU on one core and the task-graph (Alg 11) waves on
    all cores, each the median of `repeat` runs, in a child process with one BLAS thread."""
    geom, n, eps = ORACLE_SAMPLE[workload]
    cfg = W.WORKLOADS[workload]
    cores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "oracle.cpu_baseline", "--geometry", geom, "--n", str(n), "--seed",
           str(cfg["seed"]), "--eps", str(eps), "--leaf", str(cfg["leaf"]), "--eta", str(cfg["eta"]),
           "--rank-cap", str(cfg["rank_cap"]), "--repeat", str(repeat), "--threads", str(cores)]
    if not parallel:
        cmd.append("--no-parallel")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_record(o, full_model_gflop):
    """cpu_baseline of the bench line: the serial oracle's model GFLOP/s on the sample, applied
    to the model flops of one full-size factorization (seconds, the metric's unit)."""
    ser = o["serial"]
    rec = {"value": full_model_gflop / ser["gflops"] if full_model_gflop else ser["seconds"], "unit": "s",
           "cores": 1, "kind": "oracle",
           "sample": f"recursive FP64 oracle H-LU of the n={o['n']} {o['geometry']} sample (eps {o['eps']}, "
                     f"leaf 64, eta 2, cap 64), median of {len(ser['all_seconds'])}: {ser['seconds']:.2f} s "
                     f"= {ser['gflops']:.2f} model GFLOP/s on 1 core; value = the full workload's "
                     f"{full_model_gflop:.0f} model GFLOP at that rate" if full_model_gflop else
                     f"recursive FP64 oracle H-LU of the n={o['n']} {o['geometry']} sample, {ser['seconds']:.2f} s",
           "serial": {k: ser[k] for k in ("seconds", "model_gflop", "gflops", "cores", "rel_error")}}
    if "parallel" in o:
        par = o["parallel"]
        rec["parallel"] = {k: par[k] for k in ("seconds", "model_gflop", "gflops", "cores", "rel_error", "waves",
                                               "tasks")}
        rec["parallel"]["note"] = ("task-graph levels on a thread pool; the oracle's per-task work is "
                                   "Python-bound (GIL), so more threads do not speed it up")
    return rec


def run_reference(args, rank):
    if rank != 0:
        return 0
    cfg = W.WORKLOADS[args.workload]
    full = cfg.get("model_gflop")
    t0 = time.perf_counter()
    o = cpu_oracle_sample(args.workload, repeat=max(args.steps, 1), parallel=False)
    wall = time.perf_counter() - t0
    cb = cpu_baseline_record(o, full)
    line = {"metric": METRIC.format(w=args.workload), "value": cb["value"],
            "unit": "s", "impl": "reference", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(args.steps, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "sample": cb["sample"]},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def replica_points(cfg, rank):
    """Points of this rank's replica: every rank factors its own instance (seed + rank)."""
    return W.points_for(cfg["geometry"], cfg["n"], cfg["seed"] + rank)


def aggregate_ranks(total_ms, flops, dist, device):
    """Whole-job figures over the ranks: the slowest rank's time and the sum of every rank's
    FLOPs (replicas only: no data moves between ranks besides these two numbers)."""
    if dist is None:
        return total_ms, flops
    import torch
    t = torch.tensor([total_ms, flops], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


def run_batch(args, rank):
    """Batching workload: independent ellipsoid instances (n log-uniform in [4096, 65536], eps
    1e-6) factored by one hm_lu_batch call (waves of all instances merged into one launch per
    kernel kind and phase) against the same instances factored one by one with hm_lu. Seconds
    of the whole set (device time, CUDA events); the batched factors are checked for 10 eps."""
    import torch

    import paper_1911_07531_gb300 as hm
    if rank != 0:
        return 0
    hm.build_library()
    ctx = hm.HMContext(0)
    inst = W.ellipsoid_instances(count=args.instances)
    eps = 1e-6
    t0 = time.perf_counter()
    mats = [hm.hm_build(ctx, p, 64, 2.0, eps, 64) for _, p in inst]
    build_s = time.perf_counter() - t0
    stream = ctx.stream

    def timed(fn):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        a0.record(stream)
        out = fn()
        a1.record(stream)
        a1.synchronize()
        return out, a0.elapsed_time(a1) * 1e-3, time.perf_counter() - w0

    # one by one (first a warm-up pass that builds every task graph and plan)
    for A in mats:
        hm.hm_lu(ctx, A, precision=args.precision).free()

    def solo():
        tot = 0.0
        for A in mats:
            F = hm.hm_lu(ctx, A, precision=args.precision)
            tot += F.stats()["launches"]
            F.free()
        return tot
    solo_launches, solo_s, solo_wall = timed(solo)
    # batched: every call plans the merged waves on the host, uploads the plan and runs the groups
    # (instances that fit the free device memory together); the device time of the groups is
    # reported apart from the wall time of the call
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    Fs = hm.hm_lu_batch(ctx, mats, precision=args.precision)
    first_wall = time.perf_counter() - t0
    for F in Fs:
        F.free()
    torch.cuda.empty_cache()
    Fs, batch_s, batch_wall = timed(lambda: hm.hm_lu_batch(ctx, mats, precision=args.precision))
    st = Fs[0].stats()
    groups = {}
    for F in Fs:
        fs = F.stats()
        groups[(fs["seconds"], fs["launches"])] = fs["plan_seconds"]
    device_s = sum(g[0] for g in groups)
    plan_s = sum(groups.values())
    # accuracy of every batched factor: ||(A - P L U) X|| / ||A X|| on 4 Gaussian columns
    worst = 0.0
    for (n, _), A, F in zip(inst, mats, Fs):
        X = torch.randn(4, n, dtype=torch.float64, device="cuda").t()
        Ax = hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, X)
        LUx = hm.hm_matvec(ctx, A, hm.HM_OP_LU, X, F=F)
        worst = max(worst, float(torch.linalg.norm(Ax - LUx) / torch.linalg.norm(Ax)))
    for F in Fs:
        F.free()
    ns = [n for n, _ in inst]
    line = {"metric": "H-LU of the batching workload: seconds for all instances", "value": device_s, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f64" if args.precision == 0 else "f64+tf32x3",
            "data": "synthetic",
            "config": {"workload": f"{len(ns)} ellipsoid instances, n log-uniform in [4096, 65536] (seed 41), "
                                   f"1/(4pi(r+h)), leaf 64, eta 2, eps {eps}, rank cap 64",
                       "points": int(sum(ns)), "n_min": min(ns), "n_max": max(ns)},
            "batched": {"device_s": device_s, "groups": len(groups), "host_plan_s": plan_s, "call_s": batch_s,
                        "wall_s": batch_wall,
                        "launches": int(sum(g[1] for g in groups)), "first_call_wall_s": first_wall,
                        "max_rel_error": worst},
            "one_by_one": {"seconds": solo_s, "wall_s": solo_wall, "launches": int(solo_launches)},
            "speedup_device": solo_s / device_s, "speedup_call": solo_s / batch_s, "build_s": build_s}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args, rank):
    """Serving workload: the Poisson request stream (200 requests/s; n log-uniform in [2048,
    131072]; 1-32 right-hand sides; eps 1e-4 or 1e-6; half of the requests repeat solves on
    resident factors) served by the continuous-batching loop under a 150 GB budget; latency
    percentiles and served throughput."""
    if rank != 0:
        return 0
    import paper_1911_07531_gb300 as hm
    from paper_1911_07531_gb300.serve import GpuExecutor, Server, latency_summary
    hm.build_library()
    rq = W.serving_requests(count=args.requests, rate=200.0, seed=51)
    srv = Server(GpuExecutor(args.slots, precision=args.precision), slots=args.slots, budget_bytes=150e9,
                 batch=args.serve_batch)
    t0 = time.perf_counter()
    recs = srv.run(rq)
    wall = time.perf_counter() - t0
    out = latency_summary(recs)
    kinds = {}
    for r in recs:
        kinds.setdefault(r["kind"], []).append(r["latency"])
    by_kind = {k: {"count": len(v), "p50_s": float(np.percentile(v, 50)), "p99_s": float(np.percentile(v, 99))}
               for k, v in kinds.items()}
    service = np.array([r["end"] - r["start"] for r in recs])
    out["service_p50_s"] = float(np.percentile(service, 50))
    out["service_p99_s"] = float(np.percentile(service, 99))
    srv.release_all()
    line = {"metric": "serving: p50 / p99 latency and served requests per second", "value": out["p50_s"],
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.requests} requests, Poisson 200/s, sphere/cube, n log-uniform in "
                                   "[2048, 131072], 1-32 RHS, eps 1e-4 / 1e-6, 50% repeat solves (seed 51)",
                       "slots": args.slots, "budget_gb": 150, "batch": args.serve_batch},
            "latency": out, "by_kind": by_kind, "wall_s": wall, "evictions": srv.evictions,
            "factorizations_merged": int(sum(1 for r in recs if r.get("batched", 1) > 1)),
            "peak_gb": srv.peak / 1e9}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="cube131072", choices=sorted(W.WORKLOADS) + ["batch64", "serve"])
    ap.add_argument("--instances", type=int, default=64, help="batch64: number of ellipsoid instances")
    ap.add_argument("--requests", type=int, default=2000, help="serve: requests of the stream")
    ap.add_argument("--slots", type=int, default=4, help="serve: concurrent requests")
    ap.add_argument("--precision", type=int, default=0, help="batch64 / serve: HM_PREC_* of hm_lu")
    ap.add_argument("--serve-batch", type=int, default=4,
                    help="serve: waiting factorizations merged into one hm_lu_batch call")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solves", type=int, default=10)
    ap.add_argument("--no-refined", action="store_true", help="skip the eps = 1e-4 + refinement run")
    ap.add_argument("--autotune", action="store_true",
                    help="before timing, pick the GEMM split target with hm_autotune_gemm on the workload")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.workload in ("batch64", "serve"):
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the oracle has no batched or serving "
                                  "mode; its per-instance rate is the cube131072 reference line"}), flush=True)
            return 0
        return run_reference(args, rank)
    if args.workload == "batch64":
        return run_batch(args, rank)
    if args.workload == "serve":
        return run_serve(args, rank)

    import torch
    import paper_1911_07531_gb300 as hm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    hm.build_library()
    cfg = W.WORKLOADS[args.workload]
    n = cfg["n"]
    pts = replica_points(cfg, rank)
    ctx = hm.HMContext(local)
    stream = ctx.stream

    A = hm.hm_build(ctx, pts, cfg["leaf"], cfg["eta"], cfg["eps"], cfg["rank_cap"])
    tuning = None
    if args.autotune:
        best, times = hm.hm_autotune_gemm(ctx, A)
        tuning = {"gemm_work": best, "seconds_by_candidate": times}
    # warm-up (the first hm_lu also builds the task graph and the wave plan on the host)
    for _ in range(max(args.warmup, 0)):
        F = hm.hm_lu(ctx, A)
        F.free()
    st0 = A.stats()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    flops, step_ms, launches = [], [], 0
    last = None
    barrier()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        # NVTX range around the timed steps: ncu --nvtx --nvtx-include "hlu_timed/" captures them
        torch.cuda.nvtx.range_push("hlu_timed")
        for _ in range(args.steps):
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            F = hm.hm_lu(ctx, A)
            s1.record(stream)
            s1.synchronize()
            step_ms.append(s0.elapsed_time(s1))
            fs = F.stats()
            flops.append(sum(fs["flops"][:4]))
            launches += fs["launches"]
            if last is not None:
                last.free()
            last = F
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        barrier()
        wall = time.perf_counter() - t_wall0
    total_ms = e0.elapsed_time(e1)
    total_ms_max, all_flops = aggregate_ranks(total_ms, sum(flops), dist, "cuda")
    # whole job: `world` factorizations per step in the slowest replica's step time
    value = total_ms_max * 1e-3 / max(args.steps, 1) / world
    model_gflops = all_flops / (total_ms_max * 1e-3) * 1e-9
    fstats = last.stats()

    # one profiled step: per-kernel-kind device time for the roofline of the dominant kernel
    ctx.set_profiling(True)
    Fp = hm.hm_lu(ctx, A)
    ctx.set_profiling(False)
    ps = Fp.stats()
    Fp.free()
    kind_ms = dict(zip(KINDS, ps["kind_ms"]))
    kind_fl = dict(zip(KINDS, ps["kind_flops"]))
    kind_n = dict(zip(KINDS, ps["kind_launches"]))
    dom = max(KINDS, key=lambda k: kind_ms[k])
    achieved = kind_fl[dom] / (kind_ms[dom] * 1e-3) * 1e-9 if kind_ms[dom] > 0 else 0.0
    traffic = None
    if dom in PROFILED_BYTES_PER_FLOP and kind_n[dom] > 0:
        traffic = PROFILED_BYTES_PER_FLOP[dom] * kind_fl[dom] / kind_n[dom]
    roofline = {"bound": "alu", "kernel": f"k_{dom}", "achieved": achieved, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic,
                "traffic_basis": "bytes per launch: ncu DRAM bytes/FLOP summed over the kernel's launches "
                                 "in one H-LU of the n = 8192 cube (k_gemm; k_core: two launches of the "
                                 "n = 32768 sphere) x this kernel's average FLOPs per launch",
                "peak_basis": "derived FP64 DFMA peak: 152 SM x 2 FMA/clk x 2 x 2.07 GHz",
                "launches_per_step": kind_n[dom],
                "share": kind_ms[dom] / max(sum(kind_ms.values()), 1e-9),
                "per_kind_ms": {k: round(v, 3) for k, v in kind_ms.items() if v > 0},
                "per_kind_gflops": {k: round(kind_fl[k] / (kind_ms[k] * 1e-3) * 1e-9, 1)
                                    for k in KINDS if kind_ms[k] > 0}}

    # solve latency with resident factors (1 right-hand side, device buffers)
    b = torch.from_numpy(W.gaussian_rhs(n, 1, cfg["rhs_seed"])[:, 0]).to(f"cuda:{local}")
    x = torch.empty_like(b)
    lat = []
    for i in range(args.solves + 2):
        t0 = time.perf_counter()
        hm.hm_solve(ctx, last, b, x)
        dt = time.perf_counter() - t0
        if i >= 2:
            lat.append(dt * 1e3)
    lat.sort()
    p50 = lat[len(lat) // 2] if lat else None
    p99 = lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None

    # end to end through the public API with host buffers: points -> build -> LU -> solve -> x
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bh = torch.from_numpy(W.gaussian_rhs(n, 1, cfg["rhs_seed"])[:, 0]).pin_memory()
    # the H-LU's task graph and plan are prepared on a host thread during the assembly
    A2 = hm.hm_build(ctx, pts, cfg["leaf"], cfg["eta"], cfg["eps"], cfg["rank_cap"], prepare_lu=True)
    t1 = time.perf_counter()
    F2 = hm.hm_lu(ctx, A2)
    t2 = time.perf_counter()
    bd = bh.to(f"cuda:{local}", non_blocking=True)
    xd, _ = hm.hm_solve(ctx, F2, bd)
    xh = xd.cpu()
    e2e_s = time.perf_counter() - t0
    e2e_split = {"build_s": t1 - t0, "lu_s": t2 - t1, "solve_s": e2e_s - (t2 - t0)}
    e2e_flops = sum(F2.stats()["flops"][:4])
    F2.free()
    A2.free()
    del xh

    # coarse factorization + refinement (the eps = 1e-4 + FP64 refinement mode of the workload):
    # hm_lu at eps = 1e-4, then hm_solve refines to a relative residual of 1e-10 for a
    # manufactured solution b = A_exact x*, with the residual from (a) the exact kernel (n^2
    # kernel evaluations per step) or (b) the H-matrix A_H (eps 1e-6; converges to A_H's
    # solution); each reported with its exact residual and forward error
    refined = None
    if not args.no_refined:
        xs = torch.from_numpy(W.gaussian_rhs(n, 1, cfg["rhs_seed"] + 5)[:, 0]).to(f"cuda:{local}")
        bx = hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, xs)
        bnorm = float(torch.linalg.vector_norm(bx))

        def timed(fn):
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            out = fn()
            a1.record(stream)
            a1.synchronize()
            return out, a0.elapsed_time(a1) * 1e-3

        hm.hm_lu(ctx, A, eps=1e-4).free()      # first use builds the eps = 1e-4 plans (untimed)
        F64_4, f64_s = timed(lambda: hm.hm_lu(ctx, A, eps=1e-4))
        F64_4.free()
        hm.hm_lu(ctx, A, eps=1e-4, precision=hm.HM_PREC_MIXED).free()
        F4, f_s = timed(lambda: hm.hm_lu(ctx, A, eps=1e-4, precision=hm.HM_PREC_MIXED))
        refined = {"factor_eps": 1e-4, "factor_precision": "mixed: products of Alg 1 and rebuild products in FP32",
                   "factor_s": f_s, "fp64_factor_s": f64_s,
                   "factor_model_gflop": sum(F4.stats()["flops"][:4]) * 1e-9, "refine_tol": 1e-10}
        for name, op in (("exact_residual", hm.HM_OP_EXACT), ("hmatrix_residual", hm.HM_OP_A)):
            try:
                (xr, info), s_s = timed(lambda: hm.hm_solve(ctx, F4, bx, A=A, refine_tol=1e-10, max_iter=30,
                                                            residual_op=op))
                conv = True
            except hm.HMError:
                conv = False
                xr, info, s_s = None, {"iterations": 30, "rel_residual": None}, None
            rec = {"converged": conv, "iterations": info["iterations"], "rel_residual": info["rel_residual"],
                   "solve_s": s_s, "total_s": (f_s + s_s) if s_s is not None else None}
            if xr is not None:
                r = hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, xr)
                rec["exact_rel_residual"] = float(torch.linalg.vector_norm(r - bx)) / bnorm
                rec["forward_error"] = float(torch.linalg.vector_norm(xr - xs) / torch.linalg.vector_norm(xs))
            refined[name] = rec
        F4.free()
        # the plain eps = 1e-6 factor's own solve, for the accuracy comparison
        x6, _ = hm.hm_solve(ctx, last, bx)
        refined["plain_eps_1e-6"] = {
            "exact_rel_residual": float(torch.linalg.vector_norm(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, x6) - bx))
            / bnorm, "forward_error": float(torch.linalg.vector_norm(x6 - xs) / torch.linalg.vector_norm(xs))}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_record(cpu_oracle_sample(args.workload, repeat=3), statistics.median(flops) * 1e-9)

    if rank == 0:
        line = {
            "metric": METRIC.format(w=args.workload),
            "value": value, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms_max / max(args.steps, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64",
            "precision": "FP64 storage and arithmetic; the truncation core's Jacobi sweeps run in FP32 on a "
                         "Cholesky factor of the FP64 Gram-based core (eigenvalues to ~1e-6 relative), with "
                         "FP64 factorisations, products and orthogonalisation before and after",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload],
                       "l2": "no flush: every step reads and writes 13+ GB of block values (L2 is 129 MB)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "seconds_per_factorization": statistics.median(step_ms) * 1e-3,
            "model_gflops": model_gflops,
            "model_gflop_per_factorization": statistics.median(flops) * 1e-9,
            "model": "getrf 2b^3/3, trsm m b^2, gemm 2mnk, and per low-rank update (added one at a time to "
                     "the target's rank) QR(m,K)+QR(n,K)+2K^3+21K^3+2(m+n)Kk: independent of how the plan "
                     "merges updates",
            "solves_per_s": 1e3 / statistics.mean(lat) if lat else None,
            "solve_latency_ms": {"p50": p50, "p99": p99, "nrhs": 1},
            "e2e": {"value": e2e_s, "unit": "s",
                    "h2d_bytes_per_step": int(pts.nbytes + 8 * n), "d2h_bytes_per_step": int(8 * n),
                    "model_gflops": e2e_flops / e2e_s * 1e-9, "split": e2e_split,
                    "includes": "hm_build (points H2D, trees, ACA; with prepare_lu the H-LU task graph "
                                "and plan on a host thread meanwhile) + hm_lu (execution; waits for that "
                                "thread) + hm_solve with host RHS and result"},
            "gpu_launches": launches,
            "gemm_work": hm.hm_get_gemm_work(),
            "roofline": roofline,
            "clocks": clk.summary(),
            "dag": {"tasks": st0["dag_nodes"], "edges": st0["dag_edges"], "levels": st0["dag_levels"],
                    "build_s": st0["dag_seconds"], "plan_s": st0["plan_seconds"],
                    "launches_per_step": st0["plan_launches"], "truncations": st0["plan_truncations"],
                    "scratch_gb": st0["scratch_bytes"] * 1e-9},
            "factor": {"max_rank": fstats["max_rank"], "rank_cap_hits": fstats["rank_cap_hits"],
                       "flops_by_class_gflop": [round(f * 1e-9, 3) for f in fstats["flops"][:4]]},
            "wall_s": wall,
        }
        if refined is not None:
            line["refined"] = refined
        if tuning is not None:
            line["autotune"] = tuning
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
