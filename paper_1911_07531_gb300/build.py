"""Build libhmgb300.so in-tree (sm_103a only).

Host C++ (cluster tree, block tree, task graph, planner) is compiled with g++ and without
floating-point contraction so that admissibility decisions are reproducible bit for bit;
the CUDA sources are compiled by nvcc for ``-gencode arch=compute_103a,code=sm_103a``.
Translation units are compiled in parallel, then linked into one shared library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libhmgb300.so")
GENCODE = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _stale(objs, srcs) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "hmgb300.h"))
    deps.append(__file__)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every translation unit and link libhmgb300.so; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    cu, cpp = _sources()
    if not force and not _stale(None, None):
        return LIB
    nvcc = _nvcc()
    inc = ["-I", CSRC, "-I", os.path.join(HERE, "..", "include")]
    jobs = []
    for f in cu:
        o = os.path.join(OUT_DIR, f + ".o")
        jobs.append(([nvcc, GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                      "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, f), "-o", o], o))
    for f in cpp:
        o = os.path.join(OUT_DIR, f + ".o")
        jobs.append((["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", *inc, "-c",
                      os.path.join(CSRC, f), "-o", o], o))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return cmd

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, [j[0] for j in jobs]))
    tmp = LIB + ".tmp"
    link = [nvcc, GENCODE, "-shared", "-o", tmp, *[j[1] for j in jobs], "-lcudart", "-lpthread"]
    run(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
