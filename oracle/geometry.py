"""Kernel matrix entries and the mean nearest-neighbour spacing h (oracle; test-only).

The paper's model problem is a Laplace single-layer potential on the unit sphere (§5.1,
kernel 1/|x-y|); matrix entries play no role in its experiments. The workloads here use
the regularised point kernel a_ij = 1/(4 pi (|x_i - x_j| + h)) with h the mean
nearest-neighbour distance, so that the diagonal is finite: a_ii = 1/(4 pi h).
"""
from __future__ import annotations

import math

import numpy as np


def mean_nn_spacing(points: np.ndarray, chunk: int = 1024) -> float:
    """h = (1/n) sum_i min_{j != i} |x_i - x_j|, by brute force over all pairs."""
    p = np.asarray(points, dtype=np.float64)
    n = p.shape[0]
    if n < 2:
        return 0.0
    total = 0.0
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d2 = np.zeros((e - s, n))
        for a in range(3):
            diff = p[s:e, a][:, None] - p[None, :, a]
            d2 += diff * diff
        d2[np.arange(e - s), np.arange(s, e)] = np.inf
        total += float(np.sqrt(d2.min(axis=1)).sum())
    return total / n


def kernel_block(rows: np.ndarray, cols: np.ndarray, h: float) -> np.ndarray:
    """Dense block a_ij = 1/(4 pi (|x_i - y_j| + h)) for point sets rows (m x 3), cols (n x 3)."""
    d2 = np.zeros((rows.shape[0], cols.shape[0]))
    for a in range(3):
        diff = rows[:, a][:, None] - cols[None, :, a]
        d2 += diff * diff
    return 1.0 / (4.0 * math.pi * (np.sqrt(d2) + h))


def kernel_matvec_rows(points: np.ndarray, h: float, row_idx: np.ndarray,
                       x: np.ndarray, chunk: int = 256) -> np.ndarray:
    """(A_exact x)[row_idx] by evaluating the needed rows of the kernel matrix one by one."""
    out = np.zeros((len(row_idx),) + x.shape[1:])
    for s in range(0, len(row_idx), chunk):
        r = row_idx[s:s + chunk]
        out[s:s + len(r)] = kernel_block(points[r], points, h) @ x
    return out
