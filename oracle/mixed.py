"""H-LU with the factor products in FP32 (products of low-rank and dense blocks with FP32
operands and FP32 accumulation), FP64 everywhere else: leaf LU with pivots, triangular solves and
the rounded truncation. Oracle; test-only.

This is the precision split proposed for the GPU (FP32 products, FP64 truncation core and leaf
LU, an FP64 residual for iterative refinement): it tells how much of the factorization's error
the FP32 products add at a given eps, and whether refinement in FP64 recovers the accuracy.
"""
from __future__ import annotations

import numpy as np

from .hlu import HLUFactor
from .hmatrix import Dense, LowRank

F32 = np.float32


def _f32(x):
    return np.asarray(x, dtype=F32)


class MixedHLUFactor(HLUFactor):
    def mv(self, blk, X, transpose=False):
        """Y = M_blk X (or M_blk^T X) with FP32 operands and accumulation."""
        t, s = blk.row, blk.col
        Y = np.zeros(((s if transpose else t).size, X.shape[1]), dtype=F32)
        X32 = _f32(X)
        for lf in self.bt.leaves_under(blk):
            st = self.M[lf.key]
            r0, r1 = lf.row.lo - t.lo, lf.row.hi - t.lo
            c0, c1 = lf.col.lo - s.lo, lf.col.hi - s.lo
            if isinstance(st, Dense):
                D = _f32(st.D)
                if transpose:
                    Y[c0:c1] += D.T @ X32[r0:r1]
                else:
                    Y[r0:r1] += D @ X32[c0:c1]
            elif isinstance(st, LowRank):
                U, V = _f32(st.U), _f32(st.V)
                if transpose:
                    Y[c0:c1] += V @ (U.T @ X32[r0:r1])
                else:
                    Y[r0:r1] += U @ (V.T @ X32[c0:c1])
            else:
                raise TypeError("a product reached a factored diagonal leaf")
        return Y.astype(np.float64)

    def product(self, A, B):
        sa = self.M.get(A.key) if A.is_leaf else None
        sb = self.M.get(B.key) if B.is_leaf else None
        if isinstance(sa, Dense) and isinstance(sb, Dense):
            ma, mb, mc = A.row.size, A.col.size, B.col.size
            if mb > min(ma, mc):
                P = (_f32(sa.D) @ _f32(sb.D)).astype(np.float64)
                if ma <= mc:
                    return [(0, 0, np.eye(ma), P.T)]
                return [(0, 0, P, np.eye(mc))]
        return super().product(A, B)


def refine(A, f, b, tol=1e-10, max_iter=20):
    """x with |b - A x| <= tol |b|: iterative refinement with the H-LU factors f as the
    preconditioner and the residual in FP64 (A dense, permuted order). Returns (x, steps, res)."""
    x = f.usolve(f.ct.root, f.lsolve(f.ct.root, b))
    for k in range(max_iter + 1):
        r = b - A @ x
        res = np.linalg.norm(r) / np.linalg.norm(b)
        if res <= tol:
            return x, k, res
        x = x + f.usolve(f.ct.root, f.lsolve(f.ct.root, r))
    return x, max_iter, res
