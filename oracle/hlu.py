"""Recursive FP64 H-LU (Alg 1, Alg 2, Alg 3 and the upper mirror of Alg 3). Oracle; test-only.

The factorization runs in the sequential recursive order of Alg 2 and overwrites a copy of
the H-matrix in place: diagonal leaves hold the packed LU of a partially pivoted dense LU,
blocks below the diagonal hold L, blocks above hold U.

Readings (the paper is silent on these):

* Pivoting: partial pivoting inside each diagonal leaf (LAPACK getrf: first maximal
  |a| wins), so A = P L U with P block diagonal over the leaf clusters.  Solving
  L_tt X = M applies P^T of each diagonal leaf to its rows just before the leaf's
  triangular solve; X U_tt = M needs no pivoting.
* "Special routines" of the non-recursive case of Alg 1: the product A B of two blocks of
  which at least one is a leaf is formed as low-rank pieces W Z^T on sub-blocks of the
  target -- A low-rank: (U_A, B^T V_A); B low-rank: (A U_B, V_B); both dense: the
  factor pair with the smallest inner size; one dense and the other structured: an
  identity factor on the leaf-cluster side; both structured (the target is then an
  admissible leaf): recurse into A and B and collect the pieces.  A dense target adds
  the pieces; a low-rank target stacks [U_C, W_1, ...], [V_C, Z_1, ...] and truncates
  once; a structured target receives the restriction of every piece on each of its
  leaves.
* htrsl / htrsu on a leaf block whose diagonal block is structured solve with the whole
  structured triangle (block forward substitution over its leaves); a low-rank M only
  touches U (htrsl) or V (htrsu).
"""
from __future__ import annotations

import copy

import numpy as np
import scipy.linalg as sla

from .hmatrix import Dense, DiagLU, LowRank, block_matvec, truncate


class HLUFactor:
    def __init__(self, hm, eps=None, rank_cap=None):
        self.hm = hm
        self.bt = hm.bt
        self.ct = hm.ct
        self.cl = hm.ct.clusters
        self.eps = hm.eps if eps is None else float(eps)
        self.rank_cap = hm.rank_cap if rank_cap is None else int(rank_cap)
        self.stats = copy.copy(hm.stats)
        self.stats.flops = 0.0
        self.stats.cap_hits = 0
        self.stats.truncations = 0
        self.M = copy.deepcopy(hm.store)
        self.singular = False

    # -- helpers -----------------------------------------------------------------------------
    def blk(self, t, s):
        return self.bt.get(self.cl[t] if isinstance(t, int) else t,
                           self.cl[s] if isinstance(s, int) else s)

    def mv(self, blk, X, transpose=False):
        return block_matvec(self.bt, self.M, blk, X, self.stats, transpose)

    # -- Alg 2 ----------------------------------------------------------------------------------
    def factor(self):
        self.hlu(self.ct.root)
        return self

    def leaf_lu(self, b):
        """Dense LU with partial pivoting of the diagonal leaf b (Alg 2, leaf case)."""
        D = self.M[b.key].D
        lu, piv = sla.lu_factor(D, check_finite=False)
        if np.any(np.diag(lu) == 0.0):
            self.singular = True
        self.M[b.key] = DiagLU(lu, piv)
        nb = D.shape[0]
        self.stats.flops += 2.0 * nb ** 3 / 3.0

    def hlu(self, t):
        b = self.bt.get(t, t)
        if b.is_leaf:
            self.leaf_lu(b)
            return
        t0, t1 = t.sons
        self.hlu(t0)
        self.htrsu(t0, t1)
        self.htrsl(t0, t1)
        self.hmul(-1.0, self.bt.get(t1, t0), self.bt.get(t0, t1), self.bt.get(t1, t1))
        self.hlu(t1)

    # -- Alg 3: L_tt X_ts = M_ts -----------------------------------------------------------------
    def leaf_trsl(self, t, b):
        """L_tt X = M for the leaf block b = (t, s) (Alg 3, leaf case)."""
        st = self.M[b.key]
        if isinstance(st, Dense):
            st.D = self.lsolve(t, st.D)
        else:
            st.U = self.lsolve(t, st.U)

    def htrsl(self, t, s):
        b = self.bt.get(t, s)
        if b.is_leaf:
            self.leaf_trsl(t, b)
            return
        t0, t1 = t.sons
        s0, s1 = s.sons
        self.htrsl(t0, s0)
        self.htrsl(t0, s1)
        self.hmul(-1.0, self.bt.get(t1, t0), self.bt.get(t0, s0), self.bt.get(t1, s0))
        self.hmul(-1.0, self.bt.get(t1, t0), self.bt.get(t0, s1), self.bt.get(t1, s1))
        self.htrsl(t1, s0)
        self.htrsl(t1, s1)

    # -- upper mirror of Alg 3: X_st U_tt = M_st ---------------------------------------------
    def leaf_trsu(self, t, b):
        """X U_tt = M for the leaf block b = (s, t) (upper mirror of Alg 3, leaf case)."""
        st = self.M[b.key]
        if isinstance(st, Dense):
            st.D = np.ascontiguousarray(self.utsolve(t, st.D.T).T)
        else:
            st.V = self.utsolve(t, st.V)

    def htrsu(self, t, s):
        b = self.bt.get(s, t)
        if b.is_leaf:
            self.leaf_trsu(t, b)
            return
        t0, t1 = t.sons
        s0, s1 = s.sons
        self.htrsu(t0, s0)
        self.htrsu(t0, s1)
        self.hmul(-1.0, self.bt.get(s0, t0), self.bt.get(t0, t1), self.bt.get(s0, t1))
        self.hmul(-1.0, self.bt.get(s1, t0), self.bt.get(t0, t1), self.bt.get(s1, t1))
        self.htrsu(t1, s0)
        self.htrsu(t1, s1)

    # -- structured triangular solves with a thin dense right-hand side ---------------------
    def lsolve(self, t, R):
        """Y = L_tt^{-1} P_tt^T R by block forward substitution over the leaves of (t, t)."""
        R = np.array(R, dtype=np.float64, copy=True)
        b = self.bt.get(t, t)
        if b.is_leaf:
            st = self.M[b.key]
            for i, p in enumerate(st.piv):
                if p != i:
                    R[[i, p]] = R[[p, i]]
            nb = st.LU.shape[0]
            self.stats.flops += float(R.shape[1]) * nb * nb
            return sla.solve_triangular(st.LU, R, lower=True, unit_diagonal=True,
                                        check_finite=False)
        t0, t1 = t.sons
        n0 = t0.size
        R[:n0] = self.lsolve(t0, R[:n0])
        R[n0:] -= self.mv(self.bt.get(t1, t0), R[:n0])
        R[n0:] = self.lsolve(t1, R[n0:])
        return R

    def utsolve(self, t, R):
        """Y = U_tt^{-T} R (forward substitution with U^T)."""
        R = np.array(R, dtype=np.float64, copy=True)
        b = self.bt.get(t, t)
        if b.is_leaf:
            st = self.M[b.key]
            nb = st.LU.shape[0]
            self.stats.flops += float(R.shape[1]) * nb * nb
            return sla.solve_triangular(st.LU, R, lower=False, trans="T", check_finite=False)
        t0, t1 = t.sons
        n0 = t0.size
        R[:n0] = self.utsolve(t0, R[:n0])
        R[n0:] -= self.mv(self.bt.get(t0, t1), R[:n0], transpose=True)
        R[n0:] = self.utsolve(t1, R[n0:])
        return R

    def usolve(self, t, R):
        """Y = U_tt^{-1} R (backward substitution)."""
        R = np.array(R, dtype=np.float64, copy=True)
        b = self.bt.get(t, t)
        if b.is_leaf:
            st = self.M[b.key]
            nb = st.LU.shape[0]
            self.stats.flops += float(R.shape[1]) * nb * nb
            return sla.solve_triangular(st.LU, R, lower=False, check_finite=False)
        t0, t1 = t.sons
        n0 = t0.size
        R[n0:] = self.usolve(t1, R[n0:])
        R[:n0] -= self.mv(self.bt.get(t0, t1), R[n0:])
        R[:n0] = self.usolve(t0, R[:n0])
        return R

    # -- Alg 1 --------------------------------------------------------------------------------
    def hmul(self, alpha, A, B, C):
        if not (A.is_leaf or B.is_leaf or C.is_leaf):
            for i in range(2):
                for j in range(2):
                    for l in range(2):
                        self.hmul(alpha, A.sons[i][l], B.sons[l][j], C.sons[i][j])
            return
        pieces = self.product(A, B)
        if C.is_leaf:
            self.apply_to_leaf(C, alpha, pieces, C.row.lo, C.col.lo)
        else:
            for lf in self.bt.leaves_under(C):
                self.apply_to_leaf(lf, alpha, pieces, C.row.lo, C.col.lo)

    def product(self, A, B):
        """A_ab B_bc as a list of pieces (row offset, col offset, W, Z) relative to (a, c)."""
        sa, sb = self.M.get(A.key) if A.is_leaf else None, self.M.get(B.key) if B.is_leaf else None
        a, b, c = A.row, A.col, B.col
        if isinstance(sa, LowRank):
            Z = self.mv(B, sa.V, transpose=True)
            return [(0, 0, sa.U, Z)]
        if isinstance(sb, LowRank):
            W = self.mv(A, sb.U)
            return [(0, 0, W, sb.V)]
        if isinstance(sa, Dense) and isinstance(sb, Dense):
            ma, mb, mc = a.size, b.size, c.size
            if mb <= min(ma, mc):
                return [(0, 0, sa.D, sb.D.T)]
            P = sa.D @ sb.D
            self.stats.flops += 2.0 * ma * mb * mc
            if ma <= mc:
                return [(0, 0, np.eye(ma), P.T)]
            return [(0, 0, P, np.eye(mc))]
        if isinstance(sa, Dense):
            Z = self.mv(B, np.ascontiguousarray(sa.D.T), transpose=True)
            return [(0, 0, np.eye(a.size), Z)]
        if isinstance(sb, Dense):
            W = self.mv(A, sb.D)
            return [(0, 0, W, np.eye(c.size))]
        out = []
        for i in range(2):
            for j in range(2):
                for l in range(2):
                    Ai, Bj = A.sons[i][l], B.sons[l][j]
                    ro = Ai.row.lo - a.lo
                    co = Bj.col.lo - c.lo
                    for (r0, c0, W, Z) in self.product(Ai, Bj):
                        out.append((ro + r0, co + c0, W, Z))
        return out

    def apply_to_leaf(self, leaf, alpha, pieces, base_row, base_col):
        """leaf += alpha * sum of the pieces' restrictions (pieces are relative to base)."""
        lr0, lr1 = leaf.row.lo - base_row, leaf.row.hi - base_row
        lc0, lc1 = leaf.col.lo - base_col, leaf.col.hi - base_col
        m, n = lr1 - lr0, lc1 - lc0
        restricted = []
        for (r0, c0, W, Z) in pieces:
            r1, c1 = r0 + W.shape[0], c0 + Z.shape[0]
            ir0, ir1 = max(r0, lr0), min(r1, lr1)
            ic0, ic1 = max(c0, lc0), min(c1, lc1)
            if ir0 >= ir1 or ic0 >= ic1:
                continue
            restricted.append((ir0 - lr0, ic0 - lc0, W[ir0 - r0:ir1 - r0], Z[ic0 - c0:ic1 - c0]))
        if not restricted:
            return
        st = self.M[leaf.key]
        if isinstance(st, Dense):
            for (r0, c0, W, Z) in restricted:
                st.D[r0:r0 + W.shape[0], c0:c0 + Z.shape[0]] += alpha * (W @ Z.T)
                self.stats.flops += 2.0 * W.shape[0] * Z.shape[0] * W.shape[1]
            return
        Ws, Zs = [st.U], [st.V]
        for (r0, c0, W, Z) in restricted:
            Wp = np.zeros((m, W.shape[1]))
            Zp = np.zeros((n, Z.shape[1]))
            Wp[r0:r0 + W.shape[0]] = alpha * W
            Zp[c0:c0 + Z.shape[0]] = Z
            Ws.append(Wp)
            Zs.append(Zp)
        U, V = truncate(np.hstack(Ws), np.hstack(Zs), self.eps, self.rank_cap, self.stats)
        st.U, st.V = U, V

    # -- solve, matvec -------------------------------------------------------------------------
    def solve(self, b):
        """x with (P L U) x = b for b in ORIGINAL point order (n or n x nrhs)."""
        perm = self.ct.perm
        b2 = np.asarray(b, dtype=np.float64)
        vec = b2.ndim == 1
        B = b2.reshape(len(b2), -1)[perm]
        Y = self.lsolve(self.ct.root, B)
        X = self.usolve(self.ct.root, Y)
        out = np.empty_like(X)
        out[perm] = X
        return out[:, 0] if vec else out

    def apply_lu(self, x):
        """b = (P L U) x in permuted order, applying the stored factors leaf by leaf."""
        X = np.asarray(x, dtype=np.float64).reshape(x.shape[0], -1)
        n = X.shape[0]
        Z = np.zeros_like(X)
        B = np.zeros_like(X)
        for lf in self.bt.leaves():
            st = self.M[lf.key]
            r0, r1, c0, c1 = lf.row.lo, lf.row.hi, lf.col.lo, lf.col.hi
            if isinstance(st, DiagLU):
                Z[r0:r1] += np.triu(st.LU) @ X[c0:c1]
            elif r0 < c0:
                Z[r0:r1] += _leaf_apply(st, X[c0:c1])
        for lf in self.bt.leaves():
            st = self.M[lf.key]
            r0, r1, c0, c1 = lf.row.lo, lf.row.hi, lf.col.lo, lf.col.hi
            if isinstance(st, DiagLU):
                w = np.tril(st.LU, -1) @ Z[c0:c1] + Z[c0:c1]
                for i in range(len(st.piv) - 1, -1, -1):
                    p = st.piv[i]
                    if p != i:
                        w[[i, p]] = w[[p, i]]
                B[r0:r1] += w
            elif r0 > c0:
                B[r0:r1] += _leaf_apply(st, Z[c0:c1])
        assert B.shape[0] == n
        return B


def _leaf_apply(st, X):
    if isinstance(st, Dense):
        return st.D @ X
    return st.U @ (st.V.T @ X)


def hmatrix_matvec(hm, x):
    """y = A_H x in ORIGINAL order for the compressed (unfactored) H-matrix."""
    perm = hm.ct.perm
    X = np.asarray(x, dtype=np.float64).reshape(len(x), -1)[perm]
    Y = np.zeros_like(X)
    for lf in hm.bt.leaves():
        st = hm.store[lf.key]
        Y[lf.row.lo:lf.row.hi] += _leaf_apply(st, X[lf.col.lo:lf.col.hi])
    out = np.empty_like(Y)
    out[perm] = Y
    return out[:, 0] if np.ndim(x) == 1 else out
