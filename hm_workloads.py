"""Seeded synthetic inputs for the H-LU workloads (point clouds and right-hand sides).

This module holds no arithmetic of the method itself: it only draws point clouds and
random vectors. Both the FP64 oracle (``oracle/``) and the CUDA library's tests and
benchmark import it, so that both sides see exactly the same inputs.

Workloads (all seeded with ``numpy.random.default_rng`` / PCG64):

* ``fibonacci_sphere``: Fibonacci lattice on the unit sphere, z_i = 1-(2i+1)/n,
  phi_i = i*pi*(3-sqrt(5)), plus ``jitter``*N(0,1) per coordinate, then renormalised to
  |x| = 1.  Stands in for the paper's Laplace single-layer BEM on the unit sphere (§5.1);
  its Galerkin matrix is replaced by a point kernel (no quadrature), so only the block
  structure is comparable.
* ``cube_surface``: uniform on the surface of [0,1]^3 (face uniform in 1..6, then uniform
  inside the face).
* ``ellipsoid``: the jittered Fibonacci sphere scaled by axes drawn uniform in [0.5, 2]
  (not area-uniform).
* ``line_points``: n points evenly spaced on the x axis; a deterministic geometry whose
  bisection halves exactly, used for the small task-graph pins of Fig. 3 and Fig. 4.
* ``gaussian_rhs``: N(0,1) right-hand sides, column-major n x nrhs.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "fibonacci_sphere",
    "cube_surface",
    "ellipsoid",
    "line_points",
    "gaussian_rhs",
    "WORKLOADS",
    "points_for",
]


def fibonacci_sphere(n: int, seed: int, jitter: float = 1e-3) -> np.ndarray:
    """n x 3 points on the unit sphere (Fibonacci lattice + seeded jitter, renormalised)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * (math.pi * (3.0 - math.sqrt(5.0)))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    p = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    if jitter:
        rng = np.random.default_rng(seed)
        p = p + jitter * rng.standard_normal((n, 3))
        p = p / np.linalg.norm(p, axis=1, keepdims=True)
    return np.ascontiguousarray(p, dtype=np.float64)


def cube_surface(n: int, seed: int) -> np.ndarray:
    """n x 3 points uniform on the surface of the unit cube [0,1]^3."""
    rng = np.random.default_rng(seed)
    face = rng.integers(0, 6, size=n)
    uv = rng.random((n, 2))
    p = np.empty((n, 3), dtype=np.float64)
    axis = face // 2
    val = (face % 2).astype(np.float64)
    for a in range(3):
        others = [b for b in range(3) if b != a]
        sel = axis == a
        p[sel, a] = val[sel]
        p[sel, others[0]] = uv[sel, 0]
        p[sel, others[1]] = uv[sel, 1]
    return np.ascontiguousarray(p)


def ellipsoid(n: int, seed: int) -> np.ndarray:
    """n x 3 points on a random ellipsoid (axes uniform in [0.5, 2])."""
    rng = np.random.default_rng(seed)
    axes = rng.uniform(0.5, 2.0, size=3)
    p = fibonacci_sphere(n, seed + 7919) * axes[None, :]
    return np.ascontiguousarray(p)


def ellipsoid_instances(count: int = 64, seed: int = 41, n_min: int = 4096, n_max: int = 65536) -> list:
    """Independent problems of the batching workload: n log-uniform in [n_min, n_max] (rounded),
    each a seeded random ellipsoid surface (``ellipsoid``); returns [(n, points), ...]."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=count))).astype(int)
    return [(int(n), ellipsoid(int(n), seed * 1000 + i)) for i, n in enumerate(ns)]


def serving_requests(count: int = 2000, rate: float = 200.0, seed: int = 51, n_min: int = 2048,
                     n_max: int = 131072, repeat_fraction: float = 0.5) -> list:
    """The request stream of the serving workload: Poisson arrivals at `rate` per second; a
    request either factors and solves a new problem (sphere or cube 50/50, n log-uniform in
    [n_min, n_max], eps 1e-4 or 1e-6 50/50) or, with probability `repeat_fraction` once a factor
    exists, solves again with an earlier problem's factor; 1..32 right-hand sides (uniform).
    Returns dicts with rid, arrival (s), geometry, n, eps, nrhs, seed (points), rhs_seed and
    repeat_of (the rid whose factor is reused, or None)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    firsts = []
    for rid in range(count):
        t += float(rng.exponential(1.0 / rate))
        nrhs = int(rng.integers(1, 33))
        if firsts and rng.random() < repeat_fraction:
            src = out[firsts[int(rng.integers(0, len(firsts)))]]
            out.append(dict(rid=rid, arrival=t, geometry=src["geometry"], n=src["n"], eps=src["eps"], nrhs=nrhs,
                            seed=src["seed"], rhs_seed=seed * 100000 + rid, repeat_of=src["rid"]))
            continue
        n = int(np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        out.append(dict(rid=rid, arrival=t, geometry="sphere" if rng.random() < 0.5 else "cube", n=n,
                        eps=1e-4 if rng.random() < 0.5 else 1e-6, nrhs=nrhs, seed=seed * 100000 + rid,
                        rhs_seed=seed * 100000 + 50000 + rid, repeat_of=None))
        firsts.append(rid)
    return out


def line_points(n: int) -> np.ndarray:
    """n points evenly spaced on [0,1] along the x axis (exact halving under bisection)."""
    p = np.zeros((n, 3), dtype=np.float64)
    p[:, 0] = (np.arange(n, dtype=np.float64) + 0.5) / n
    return p


def gaussian_rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Column-major (Fortran-ordered) n x nrhs N(0,1) right-hand sides."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, nrhs)))


# The workloads of the benchmark configurations; seed convention: config c uses 10c+1 for
# points and 10c+2 for right-hand sides.
WORKLOADS = {
    "sphere2048": dict(geometry="sphere", n=2048, seed=11, rhs_seed=12, leaf=64, eta=2.0,
                       eps=1e-4, rank_cap=64),
    "sphere8192": dict(geometry="sphere", n=8192, seed=21, rhs_seed=22, leaf=64, eta=2.0,
                       eps=1e-6, rank_cap=64),
    "sphere32768": dict(geometry="sphere", n=32768, seed=21, rhs_seed=22, leaf=64, eta=2.0,
                        eps=1e-6, rank_cap=64),
    "cube131072": dict(geometry="cube", n=131072, seed=31, rhs_seed=32, leaf=64, eta=2.0,
                       eps=1e-6, rank_cap=64,
                       # model GFLOP of one factorization of this matrix (getrf, trsm, gemm and the
                       # per-update truncation model, with the ranks the factorization realises);
                       # scales the oracle's timed sample to this size in the benchmark's CPU baseline
                       model_gflop=2274.08),
}


def points_for(geometry: str, n: int, seed: int) -> np.ndarray:
    if geometry == "sphere":
        return fibonacci_sphere(n, seed)
    if geometry == "cube":
        return cube_surface(n, seed)
    if geometry == "ellipsoid":
        return ellipsoid(n, seed)
    if geometry == "line":
        return line_points(n)
    raise ValueError(f"unknown geometry {geometry!r}")
