"""Small command-line runs of the library on the seeded workloads, for profilers and timing.

  python -m paper_1911_07531_gb300.run_case lu GEOMETRY N EPS PRECISION
      builds the H-matrix of the points of `hm_workloads` (seed 31, leaf 64, eta 2, rank cap 64)
      and runs one hm_lu with HM_PREC_* = PRECISION inside the NVTX range "hm_lu"; prints its
      device seconds, launches and FLOPs per kernel kind as a JSON line.
  python -m paper_1911_07531_gb300.run_case xmv N
      the cube matrix at eps 1e-6 and two exact-kernel matvecs (HM_OP_EXACT) of one vector.
  python -m paper_1911_07531_gb300.run_case overlap WORKLOAD EPS REPEATS
      hm_lu of a workload with the wave overlap off and on (hm_set_overlap), alternating, after
      a warm-up of each; prints the device seconds of every factorization as JSON lines.
  python -m paper_1911_07531_gb300.run_case accumulate WORKLOAD EPS REPEATS
      hm_lu of a workload as the H-LU of Alg 2 and as the accumulator H-LU, alternating, after a
      warm-up of each; prints device seconds, rounded additions and the arena size as JSON lines.
  python -m paper_1911_07531_gb300.run_case kinds WORKLOAD EPS
      one hm_lu per precision (FP64, MIXED, MIXED_TC) of a workload of `hm_workloads.WORKLOADS`
      after a warm-up, then a profiled one (CUDA events around every launch); prints the device
      milliseconds per kernel kind as JSON lines. With HMGB300_LAUNCH_LOG=<prefix> every profiled
      launch is written to <prefix>_<precision>.csv.
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KINDS = ("getrf", "trsm", "gemm", "copy", "stack", "core", "eval", "aca")


def _lu(geom, n, eps, prec):
    import torch

    import hm_workloads as W

    from . import HMContext, build_library, hm_build, hm_lu
    build_library()
    ctx = HMContext(0)
    A = hm_build(ctx, W.points_for(geom, n, 31), 64, 2.0, eps, 64)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("hm_lu")   # profilers can select the factorization's launches
    F = hm_lu(ctx, A, precision=prec)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    st = F.stats()
    print(json.dumps({"seconds": st["seconds"], "launches": st["launches"],
                      "kind_flops": dict(zip(KINDS, st["kind_flops"]))}), flush=True)


def _xmv(n):
    import torch

    import hm_workloads as W

    from . import HM_OP_EXACT, HMContext, build_library, hm_build, hm_matvec
    build_library()
    ctx = HMContext(0)
    A = hm_build(ctx, W.points_for("cube", n, 31), 64, 2.0, 1e-6, 64)
    x = torch.randn(n, dtype=torch.float64, device=f"cuda:{ctx.device}")
    for _ in range(2):
        y = hm_matvec(ctx, A, HM_OP_EXACT, x)
    torch.cuda.synchronize()
    print("ok", float(y.norm()))


def _kinds(workload, eps):
    import hm_workloads as W

    from . import HMContext, build_library, hm_build, hm_lu
    build_library()
    w = W.WORKLOADS[workload]
    ctx = HMContext(0)
    A = hm_build(ctx, W.points_for(w["geometry"], w["n"], w["seed"]), w["leaf"], w["eta"], w["eps"], w["rank_cap"])
    prefix = os.environ.pop("HMGB300_LAUNCH_LOG", None)
    for prec, name in ((0, "fp64"), (1, "mixed"), (2, "mixedtc")):
        hm_lu(ctx, A, eps=eps, precision=prec).free()
        F = hm_lu(ctx, A, eps=eps, precision=prec)
        seconds = F.stats()["seconds"]
        F.free()
        if prefix:
            os.environ["HMGB300_LAUNCH_LOG"] = f"{prefix}_{name}.csv"
        ctx.set_profiling(True)
        F = hm_lu(ctx, A, eps=eps, precision=prec)
        ctx.set_profiling(False)
        os.environ.pop("HMGB300_LAUNCH_LOG", None)
        st = F.stats()
        print(json.dumps({"precision": name, "eps": eps, "seconds": seconds,
                          "kind_ms": dict(zip(KINDS, [round(v, 1) for v in st["kind_ms"]])),
                          "tc_ms": round(st["tc_ms"], 1), "f32_ms": round(st["f32_ms"], 1),
                          "launches": st["launches"]}), flush=True)
        F.free()


def _overlap(workload, eps, repeats):
    import hm_workloads as W

    from . import HMContext, build_library, hm_build, hm_lu, hm_set_overlap
    build_library()
    w = W.WORKLOADS[workload]
    ctx = HMContext(0)
    A = hm_build(ctx, W.points_for(w["geometry"], w["n"], w["seed"]), w["leaf"], w["eta"], w["eps"], w["rank_cap"])
    for on in (0, 1):
        hm_set_overlap(on)
        hm_lu(ctx, A, eps=eps).free()
    for r in range(repeats):
        for on in (0, 1):
            hm_set_overlap(on)
            F = hm_lu(ctx, A, eps=eps)
            st = F.stats()
            F.free()
            print(json.dumps({"overlap": on, "repeat": r, "seconds": st["seconds"],
                              "plan_truncations": st["plan_truncations"],
                              "plan_deferred": st["plan_deferred"]}), flush=True)


def _accumulate(workload, eps, repeats):
    import hm_workloads as W

    from . import HMContext, build_library, hm_build, hm_lu
    build_library()
    w = W.WORKLOADS[workload]
    ctx = HMContext(0)
    A = hm_build(ctx, W.points_for(w["geometry"], w["n"], w["seed"]), w["leaf"], w["eta"], w["eps"], w["rank_cap"])
    for acc in (False, True):
        hm_lu(ctx, A, eps=eps, accumulate=acc).free()
    for r in range(repeats):
        for acc in (False, True):
            F = hm_lu(ctx, A, eps=eps, accumulate=acc)
            st = F.stats()
            F.free()
            print(json.dumps({"accumulate": acc, "repeat": r, "seconds": st["seconds"],
                              "plan_seconds": st["plan_seconds"], "plan_launches": st["plan_launches"],
                              "plan_truncations": st["plan_truncations"], "arena_gb": st["arena_bytes"] / 1e9,
                              "accumulated_pieces": st["accumulated_pieces"],
                              "scratch_gb": st["scratch_bytes"] / 1e9}), flush=True)


def main(argv=None):
    a = sys.argv[1:] if argv is None else argv
    if a and a[0] == "lu" and len(a) == 5:
        _lu(a[1], int(a[2]), float(a[3]), int(a[4]))
    elif a and a[0] == "xmv" and len(a) == 2:
        _xmv(int(a[1]))
    elif a and a[0] == "overlap" and len(a) == 4:
        _overlap(a[1], float(a[2]), int(a[3]))
    elif a and a[0] == "accumulate" and len(a) == 4:
        _accumulate(a[1], float(a[2]), int(a[3]))
    elif a and a[0] == "kinds" and len(a) == 3:
        _kinds(a[1], float(a[2]))
    else:
        print(__doc__)
        return 2
    return 0


if __name__ == "__main__":
    sys.exit(main())
