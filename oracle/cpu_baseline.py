"""Times the FP64 oracle's H-LU on the host cores and prints one JSON line. Oracle; test-only.

Two variants on the same seeded H-matrix:
  serial    the recursive H-LU (Alg 2 with Alg 1, Alg 3 and its mirror), one core;
  parallel  the same arithmetic driven by the task graph (Alg 11), the tasks of each
            longest-path level on a pool of host threads (``WaveParallelHLU``).
Each is timed `repeat` times (median reported) after the H-matrix is assembled (and, for the
parallel variant, after its task graph is built); the flop count
is the oracle's model count of the factorization (getrf 2b^3/3, trsm m b^2, gemm 2mnk,
truncation QR + core + SVD + rebuild). Run it with one BLAS thread per process
(OMP_NUM_THREADS=1 and the like) so that `threads` is the number of cores the parallel variant
uses.

  python -m oracle.cpu_baseline --geometry cube --n 2048 --eps 1e-6 --repeat 3 --threads 16
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np


def main(argv=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import hm_workloads as W

    from .hlu import HLUFactor
    from .hmatrix import HMatrix
    from .wave_parallel import WaveParallelHLU

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--geometry", default="cube")
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--seed", type=int, default=31)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--eta", type=float, default=2.0)
    ap.add_argument("--rank-cap", type=int, default=64)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--no-parallel", action="store_true")
    a = ap.parse_args(argv)

    p = W.points_for(a.geometry, a.n, a.seed)
    t0 = time.perf_counter()
    hmo = HMatrix(p, a.leaf, a.eta, a.eps, a.rank_cap)
    build_s = time.perf_counter() - t0
    out = {"geometry": a.geometry, "n": a.n, "eps": a.eps, "build_s": build_s, "host_cores": os.cpu_count()}
    X = np.random.default_rng(1).standard_normal((a.n, 4))
    Ax = None
    variants = [("serial", lambda: HLUFactor(hmo), 1)]
    if not a.no_parallel:
        variants.append(("parallel", lambda: WaveParallelHLU(hmo, threads=a.threads).plan(), a.threads))
    for name, make, cores in variants:
        secs, f = [], None
        for _ in range(max(1, a.repeat)):
            f = make()
            t0 = time.perf_counter()
            f.factor()
            secs.append(time.perf_counter() - t0)
        if Ax is None and a.n <= 4096:
            A = hmo.exact_dense()
            Ax = A @ X
        err = float(np.linalg.norm(Ax - f.apply_lu(X)) / np.linalg.norm(Ax)) if Ax is not None else None
        med = statistics.median(secs)
        out[name] = {"seconds": med, "all_seconds": secs, "model_gflop": f.stats.flops * 1e-9,
                     "gflops": f.stats.flops * 1e-9 / med, "cores": cores, "rel_error": err}
        if name == "parallel":
            out[name].update(waves=f.waves, tasks=f.tasks)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
