"""Micro-op-by-micro-op execution of the library's host plans in numpy (test infrastructure).

The library expands the task graph into launches of batched micro-ops whose meaning is fixed
by their descriptors (the library's ``csrc/ops.h``). This module gives each kind that meaning
on host arrays, so that a plan exported by ``Structure.plan`` can be run on the CPU and its
data flow (addresses, strides, dynamic sizes, phase order, stacking of rounded additions)
checked against the oracle without a GPU:

  getrf  in-place LU with partial pivoting of a b x b column-major leaf, LAPACK pivots;
  trsm   x := L^-1 P^T x, U^-T x, U^-1 x, U x or P L x with a packed LU, on strided vectors;
  gemm   C (+)= alpha A B on strided operands with dynamic dimension adders; flags select
         accumulate / overwrite, an upper or unit-lower A, and an upper-triangle-only C;
  copy   zero / identity / alpha-scaled copy / alpha-scaled add of a strided block;
  stack  W = [U, a_1 W_1, ...], Z = [V, Z_1, ...] with zero rows outside each piece (without U,
         V for a temporary sum of a tree of rounded additions), the stacked rank K, and zeroed
         K x K Gram matrices;
  core   from the Gram matrices of W and Z (upper triangles): coefficient matrices T_W, T_Z
         with W T_W = U_k S_k, Z T_Z = V_k for the singular values above eps s_1 (at most
         the cap), and the new rank k. Computed here by symmetric eigendecompositions of the
         Gram matrices and an SVD of the small core, not by the kernel's algorithm;
  eval   a dense leaf 1 / (4 pi (|x_i - x_j| + h)) from the permuted points;
  aca    a low-rank approximation U V^T of an admissible leaf to the relative tolerance, at most
         kmax terms (here a truncated SVD of the evaluated block stands in for the cross
         approximation: any approximation within the tolerance is a valid result).

Every strided access is bounds-checked against its memory space, so a planner address error
fails loudly here. The oracle is not used by this module.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
from numpy.lib.stride_tricks import as_strided

MASK = (1 << 60) - 1
K_GETRF, K_TRSM, K_GEMM, K_COPY, K_STACK, K_CORE, K_EVAL, K_ACA = range(8)
GF_ATOMIC, GF_OVERWRITE, GF_A_UPPER, GF_A_UNITLOWER, GF_SYM_UPPER = 1, 2, 4, 8, 16
SP_F, SP_S, SP_X, SP_A, SP_P, SP_S2, SP_ACC = 0, 1, 2, 3, 4, 5, 6
IS_RANK, IS_PIV, IS_S, IS_ARANK, IS_S2 = 0, 1, 2, 3, 4
KMAX_ENTRIES = 256
TF_NOSELF = 1   # a stack without the output's own factors (a temporary sum of a tree of rounded additions)


class PlanSim:
    def __init__(self, sizes, nrhs_space=0):
        self.d = {SP_F: np.zeros(int(sizes["nvalues"])), SP_S: np.zeros(int(sizes["scratch_doubles"])),
                  SP_X: np.zeros(int(nrhs_space)), SP_S2: np.zeros(int(sizes["scratch_doubles"])),
                  SP_ACC: np.zeros(int(sizes["arena_doubles"]))}
        self.i = {IS_RANK: np.zeros(int(sizes["nranks"]), np.int64), IS_PIV: np.zeros(int(sizes["npiv"]), np.int64),
                  IS_S: np.zeros(max(int(sizes["scratch_ints"]), 1), np.int64),
                  IS_S2: np.zeros(max(int(sizes["scratch_ints"]), 1), np.int64)}
        self.cap_hits = 0
        self.singular = 0
        self.trace = None   # a list: every access is recorded as (table, space, element offsets)
        self.h = None   # kernel regularisation (assembly plans)

    # -- addressing ------------------------------------------------------------------------------
    def _space(self, ref, table):
        r = int(ref)
        assert r != 0, "null reference"
        return table[(r >> 60) - 1], r & MASK

    def mat(self, ref, rs, cs, m, n):
        """Writable m x n view, element (i, j) at ref + i rs + j cs."""
        arr, off = self._space(ref, self.d)
        rs, cs, m, n = int(rs), int(cs), int(m), int(n)
        assert rs >= 0 and cs >= 0 and m >= 0 and n >= 0
        if m and n:
            last = off + (m - 1) * rs + (n - 1) * cs
            assert 0 <= off and last < arr.size, f"access [{off}, {last}] outside a space of {arr.size}"
            if self.trace is not None:
                self.trace.append(("d", (int(ref) >> 60) - 1,
                                   (off + rs * np.arange(m)[:, None] + cs * np.arange(n)[None, :]).ravel()))
        return as_strided(arr[off:], shape=(m, n), strides=(rs * 8, cs * 8))

    def _itrace(self, ref, off):
        if self.trace is not None:
            self.trace.append(("i", (int(ref) >> 60) - 1, np.array([off])))

    def ival(self, ref):
        arr, off = self._space(ref, self.i)
        assert off < arr.size
        self._itrace(ref, off)
        return int(arr[off])

    def iset(self, ref, v):
        arr, off = self._space(ref, self.i)
        assert off < arr.size
        self._itrace(ref, off)
        arr[off] = v

    def dim(self, s, d):
        return int(s) + (self.ival(d) if int(d) else 0)

    # -- micro-ops ---------------------------------------------------------------------------------
    def getrf(self, op):
        b = int(op["b"])
        A = self.mat(op["A"], 1, b, b, b)
        lu, piv = sla.lu_factor(np.array(A), check_finite=False)
        self.singular += int(np.count_nonzero(np.diag(lu) == 0.0))
        A[:] = lu
        arr, off = self._space(op["piv"], self.i)
        arr[off:off + b] = piv

    def trsm(self, op):
        nv, b, mode = self.dim(op["nv"], op["nvd"]), int(op["b"]), int(op["mode"])
        if nv <= 0:
            return
        T = np.array(self.mat(op["T"], 1, b, b, b))
        X = self.mat(op["X"], op["x_es"], op["x_vs"], b, nv)
        x = np.array(X)
        L = np.tril(T, -1) + np.eye(b)
        U = np.triu(T)
        piv = None
        if int(op["piv"]):
            arr, off = self._space(op["piv"], self.i)
            piv = arr[off:off + b]
        if mode == 0:
            for r in range(b):
                p = int(piv[r])
                if p != r:
                    x[[r, p]] = x[[p, r]]
            x = sla.solve_triangular(L, x, lower=True, unit_diagonal=True)
        elif mode == 1:
            x = sla.solve_triangular(U, x, trans="T", lower=False)
        elif mode == 2:
            x = sla.solve_triangular(U, x, lower=False)
        elif mode == 3:
            x = U @ x
        else:
            x = L @ x
            for r in range(b - 1, -1, -1):
                p = int(piv[r])
                if p != r:
                    x[[r, p]] = x[[p, r]]
        X[:] = x

    def gemm(self, op):
        m, n = self.dim(op["m"], op["md"]), self.dim(op["n"], op["nd"])
        k = max(self.dim(op["k"], op["kd"]), 0)
        fl = int(op["flags"])
        overwrite = bool(fl & GF_OVERWRITE)
        if m <= 0 or n <= 0 or (k == 0 and not overwrite):
            return
        if k > 0:
            A = np.array(self.mat(op["A"], op["a_rs"], op["a_cs"], m, k))
            if fl & GF_A_UPPER:
                A = np.triu(A)
            if fl & GF_A_UNITLOWER:
                A = np.tril(A, -1) + np.eye(m, k)
            B = np.array(self.mat(op["B"], op["b_rs"], op["b_cs"], k, n))
            P = float(op["alpha"]) * (A @ B)
        else:
            P = np.zeros((m, n))
        C = self.mat(op["C"], op["c_rs"], op["c_cs"], m, n)
        sel = np.triu(np.ones((m, n), bool)) if fl & GF_SYM_UPPER else np.ones((m, n), bool)
        if overwrite:
            C[sel] = P[sel]
        else:
            C[sel] = C[sel] + P[sel]

    def copy(self, op):
        m, n, mode = self.dim(op["m"], op["md"]), self.dim(op["n"], op["nd"]), int(op["mode"])
        if m <= 0 or n <= 0:
            return
        D = self.mat(op["dst"], op["d_rs"], op["d_cs"], m, n)
        if mode == 0:
            D[:] = 0.0
        elif mode == 1:
            D[:] = np.eye(m, n)
        else:
            S = float(op["alpha"]) * np.array(self.mat(op["src"], op["s_rs"], op["s_cs"], m, n))
            if mode == 2:
                D[:] = S
            else:
                D[:] = D + S

    def stack(self, op, entries):
        m, n, Kc = int(op["m"]), int(op["n"]), int(op["Kcap"])
        kself = 0 if int(op["flags"]) & TF_NOSELF else self.ival(op["rank"])
        ent = entries[int(op["first_entry"]):int(op["first_entry"]) + min(int(op["n_entries"]), KMAX_ENTRIES)]
        ke = [max(self.dim(e["k"], e["kd"]), 0) for e in ent]
        K = min(kself + sum(ke), Kc)
        self.iset(op["Kd"], K)
        self.mat(op["Gw"], 1, Kc, K, K)[:] = 0.0
        self.mat(op["Gz"], 1, Kc, K, K)[:] = 0.0
        W = self.mat(op["Wst"], 1, m, m, Kc)
        Z = self.mat(op["Zst"], 1, n, n, Kc)
        c = min(kself, K)
        W[:, :c] = self.mat(op["U"], 1, m, m, c)
        Z[:, :c] = self.mat(op["V"], 1, n, n, c)
        for e, k in zip(ent, ke):
            k = max(0, min(k, K - c))
            if k == 0:
                continue
            W[:, c:c + k] = 0.0
            Z[:, c:c + k] = 0.0
            r0, nr, c0, nc = int(e["row_off"]), int(e["nrows"]), int(e["col_off"]), int(e["ncols"])
            W[r0:r0 + nr, c:c + k] = float(e["alpha"]) * self.mat(e["W"], e["w_rs"], e["w_cs"], nr, k)
            Z[c0:c0 + nc, c:c + k] = self.mat(e["Z"], e["z_rs"], e["z_cs"], nc, k)
            c += k

    @staticmethod
    def _gram_factor(G, tol):
        """R (r x K) and a right inverse Rinv (K x r) with G = R^T R on the numerical range."""
        lam, E = np.linalg.eigh(G)
        keep = lam > tol * max(lam.max(), 0.0)
        if not keep.any():
            return np.zeros((0, G.shape[0])), np.zeros((G.shape[0], 0))
        lam, E = lam[keep], E[:, keep]
        s = np.sqrt(lam)
        return (E * s).T, E / s

    def core(self, op):
        Kc, cap, eps = int(op["Kcap"]), int(op["cap"]), float(op["eps"])
        K = self.ival(op["Kd"])
        if K <= 0:
            self.iset(op["rank"], 0)
            return
        Gw = np.triu(np.array(self.mat(op["Gw"], 1, Kc, K, K)))
        Gz = np.triu(np.array(self.mat(op["Gz"], 1, Kc, K, K)))
        Gw = Gw + np.triu(Gw, 1).T
        Gz = Gz + np.triu(Gz, 1).T
        tol = 64 * K * np.finfo(float).eps
        Rw, Rwi = self._gram_factor(Gw, tol)
        Rz, Rzi = self._gram_factor(Gz, tol)
        k = 0
        if Rw.shape[0] and Rz.shape[0]:
            X, s, Yt = np.linalg.svd(Rw @ Rz.T)
            k = int(np.count_nonzero(s > eps * s[0])) if s[0] > 0 else 0
            if k > cap:
                self.cap_hits += 1
                k = cap
        if k:
            self.mat(op["Tw"], 1, Kc, K, k)[:] = Rwi @ (X[:, :k] * s[:k])
            self.mat(op["Tz"], 1, Kc, K, k)[:] = Rzi @ Yt[:k].T
        self.iset(op["rank"], k)

    def _block(self, r0, c0, m, n):
        P = self.d[SP_P].reshape(-1, 3)
        d = np.sqrt(((P[r0:r0 + m, None, :] - P[None, c0:c0 + n, :]) ** 2).sum(-1))
        return 1.0 / (4.0 * np.pi * (d + self.h))

    def eval(self, op):
        m, n = int(op["m"]), int(op["n"])
        self.mat(op["D"], 1, m, m, n)[:] = self._block(int(op["r0"]), int(op["c0"]), m, n)

    def aca(self, op):
        m, n, kmax, tol = int(op["m"]), int(op["n"]), int(op["kmax"]), float(op["tol"])
        X, s, Yt = np.linalg.svd(self._block(int(op["r0"]), int(op["c0"]), m, n), full_matrices=False)
        k = min(int(np.count_nonzero(s > tol * s[0])), kmax) if s[0] > 0 else 0
        self.mat(op["U"], 1, m, m, k)[:] = X[:, :k] * s[:k]
        self.mat(op["V"], 1, n, n, k)[:] = Yt[:k].T
        self.iset(op["kd"], k)

    # -- plans -------------------------------------------------------------------------------------
    @staticmethod
    def latest_order(launches):
        """The launches of an H-LU plan with side launches in the latest order the library's
        streams allow: the side launches of wave w after every other launch of wave w + 1, just
        before wave w + 2 starts (the sequential plan order is the earliest one)."""
        out, held = [], {}
        cur = None
        for ln in launches:
            w = int(ln["wave"])
            if int(ln["side"]):
                held.setdefault(w, []).append(ln)
                continue
            if w != cur:
                cur = w
                out.extend(held.pop(w - 2, []))
            out.append(ln)
        for w in sorted(held):
            out.extend(held[w])
        return out

    def run_launch(self, P, ln):
        tables = {K_GETRF: P["getrf"], K_TRSM: P["trsm"], K_GEMM: P["gemm"], K_COPY: P["copy"],
                  K_STACK: P["trunc"], K_CORE: P["trunc"], K_EVAL: P.get("eval"), K_ACA: P.get("aca")}
        fns = {K_GETRF: self.getrf, K_TRSM: self.trsm, K_GEMM: self.gemm, K_COPY: self.copy,
               K_STACK: lambda op: self.stack(op, P["entries"]), K_CORE: self.core, K_EVAL: self.eval,
               K_ACA: self.aca}
        kind, b, c = int(ln["kind"]), int(ln["begin"]), int(ln["count"])
        ops = tables[kind]
        assert b + c <= len(ops)
        for op in ops[b:b + c]:
            fns[kind](op)

    def footprint(self, P, ln):
        """Runs one launch and returns what it accessed and what it changed: two dicts
        {(table, space): sorted element offsets}, table "d" (doubles) or "i" (integers)."""
        snap = {("d", k): v.copy() for k, v in self.d.items()}
        snap.update({("i", k): v.copy() for k, v in self.i.items()})
        self.trace = []
        try:
            self.run_launch(P, ln)
        finally:
            tr, self.trace = self.trace, None
        acc = {}
        for t, sp, offs in tr:
            acc.setdefault((t, sp), []).append(offs)
        acc = {k: np.unique(np.concatenate(v)) for k, v in acc.items()}
        wr = {}
        for (t, sp), before in snap.items():
            now = (self.d if t == "d" else self.i)[sp]
            ch = np.flatnonzero(before != now)
            if ch.size:
                wr[(t, sp)] = ch
        return acc, wr

    def run(self, P, order=None):
        for ln in (P["launches"] if order is None else order):
            self.run_launch(P, ln)
        return self
