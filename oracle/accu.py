"""Accumulator-based H-LU (§2.3: Alg 4 add_upd, Alg 5 apply_upd, Alg 6 shift_upd, Alg 7 hlu and
Alg 8 htrsl with accumulators, and the upper mirror of Alg 8). Oracle; test-only.

Updates are not applied where they arise: add_upd collects the product alpha A B in the
accumulator U_{t,s} of the destination block when one of the three blocks is a leaf (the
product can then be formed), and otherwise records the triple in the pending set P_{t,s}.
Before a block is factorised or solved with, its accumulated updates are shifted down to the
sub-blocks (shift_upd) at each recursive step, and a leaf adds its accumulator once
(apply_upd) before the dense factorisation or solve.

Three accumulator formats are provided (§2.3 leaves the format open): a list of pieces
(AccuHLUFactor, the reference form used by the task runner), a factorised low-rank matrix
rounded at every addition (LowRankAccuHLUFactor), and a list of pieces compressed once per
structured block when shifted to the sons (CoarseAccuHLUFactor).

Readings (the paper leaves these open or prints them garbled):

* Storage of an accumulator: the list of its pieces W Z^T on sub-blocks of (t, s) (the paper
  leaves the format open), restricted to the sons by shift_upd; a low-rank leaf receives all
  pieces of its accumulator in one rounded addition, a dense leaf adds them.
* Products are formed exactly as in the recursive oracle (``HLUFactor.product``).
* Alg 7's update reads add_upd(-1, L_{t1,t0}, U_{t0,t1}, A_{t1,t1}); the second update of
  Alg 8 uses L_{t1,t0} (both are printed with other indices).
* Upper mirror of Alg 8 for X U_tt = M_st: shift_upd(M_st); htrsu(t0, s0), htrsu(t0, s1);
  add_upd(-1, X_{s0,t0}, U_{t0,t1}, M_{s0,t1}), add_upd(-1, X_{s1,t0}, U_{t0,t1}, M_{s1,t1});
  htrsu(t1, s0), htrsu(t1, s1); at a leaf apply_upd(M_st), then the solve.
"""
from __future__ import annotations

import numpy as np

from .hlu import HLUFactor
from .hmatrix import Dense, truncate


class AccuHLUFactor(HLUFactor):
    def __init__(self, hm, eps=None, rank_cap=None):
        super().__init__(hm, eps, rank_cap)
        self.acc = {}       # block key -> pieces (r0, c0, alpha W, Z) relative to the block
        self.pending = {}   # block key -> [(alpha, A, B)]

    # -- Alg 4 ------------------------------------------------------------------------------------
    def add_upd(self, alpha, A, B, C):
        if A.is_leaf or B.is_leaf or C.is_leaf:
            acc = self.acc.setdefault(C.key, [])
            for (r0, c0, W, Z) in self.product(A, B):
                acc.append((r0, c0, alpha * W, Z))
        else:
            self.pending.setdefault(C.key, []).append((alpha, A, B))

    # -- Alg 6 ------------------------------------------------------------------------------------
    def shift_upd(self, C):
        acc = self.acc.pop(C.key, [])
        pend = self.pending.pop(C.key, [])
        for i in range(2):
            for j in range(2):
                Cs = C.sons[i][j]
                ro, co = Cs.row.lo - C.row.lo, Cs.col.lo - C.col.lo
                m, n = Cs.row.size, Cs.col.size
                for (r0, c0, W, Z) in acc:
                    r1, c1 = r0 + W.shape[0], c0 + Z.shape[0]
                    ir0, ir1 = max(r0, ro), min(r1, ro + m)
                    ic0, ic1 = max(c0, co), min(c1, co + n)
                    if ir0 < ir1 and ic0 < ic1:
                        self.acc.setdefault(Cs.key, []).append(
                            (ir0 - ro, ic0 - co, W[ir0 - r0:ir1 - r0], Z[ic0 - c0:ic1 - c0]))
                for (alpha, A, B) in pend:
                    for l in range(2):
                        self.add_upd(alpha, A.sons[i][l], B.sons[l][j], Cs)

    # -- Alg 5 ------------------------------------------------------------------------------------
    def apply_upd(self, C):
        if not C.is_leaf:
            self.shift_upd(C)
            for i in range(2):
                for j in range(2):
                    self.apply_upd(C.sons[i][j])
            return
        acc = self.acc.pop(C.key, [])
        if acc:
            self.apply_to_leaf(C, 1.0, acc, C.row.lo, C.col.lo)

    # -- Alg 7 ------------------------------------------------------------------------------------
    def hlu(self, t):
        b = self.bt.get(t, t)
        if b.is_leaf:
            self.apply_upd(b)
            self.leaf_lu(b)
            return
        self.shift_upd(b)
        t0, t1 = t.sons
        self.hlu(t0)
        self.htrsu(t0, t1)
        self.htrsl(t0, t1)
        self.add_upd(-1.0, self.bt.get(t1, t0), self.bt.get(t0, t1), self.bt.get(t1, t1))
        self.hlu(t1)

    # -- Alg 8: L_tt X_ts = M_ts --------------------------------------------------------------------
    def htrsl(self, t, s):
        b = self.bt.get(t, s)
        if b.is_leaf:
            self.apply_upd(b)
            self.leaf_trsl(t, b)
            return
        self.shift_upd(b)
        t0, t1 = t.sons
        s0, s1 = s.sons
        self.htrsl(t0, s0)
        self.htrsl(t0, s1)
        self.add_upd(-1.0, self.bt.get(t1, t0), self.bt.get(t0, s0), self.bt.get(t1, s0))
        self.add_upd(-1.0, self.bt.get(t1, t0), self.bt.get(t0, s1), self.bt.get(t1, s1))
        self.htrsl(t1, s0)
        self.htrsl(t1, s1)

    # -- upper mirror of Alg 8: X_st U_tt = M_st ------------------------------------------------------
    def htrsu(self, t, s):
        b = self.bt.get(s, t)
        if b.is_leaf:
            self.apply_upd(b)
            self.leaf_trsu(t, b)
            return
        self.shift_upd(b)
        t0, t1 = t.sons
        s0, s1 = s.sons
        self.htrsu(t0, s0)
        self.htrsu(t0, s1)
        self.add_upd(-1.0, self.bt.get(s0, t0), self.bt.get(t0, t1), self.bt.get(s0, t1))
        self.add_upd(-1.0, self.bt.get(s1, t0), self.bt.get(t0, t1), self.bt.get(s1, t1))
        self.htrsu(t1, s0)
        self.htrsu(t1, s1)

    def factor(self):
        super().factor()
        # every collected update reached its leaf
        assert not any(self.acc.values()) and not any(self.pending.values())
        return self


class AccuTaskRunner(AccuHLUFactor):
    """Executes the tasks of the accumulator task graph (§3.2, Table 2) one at a time, in any
    order that respects the graph's edges; used to check that the graph carries every
    dependency the accumulator H-LU needs.

    Each task does its own part of Alg 4-8. add_upd ('add', t, r, s) forms the product of the
    leaf-level operands and appends it to U_ts. Accumulators are pulled down the block tree:
    shift_upd ('shift', t, s) appends the restriction of the parent's accumulator to U_ts, and
    apply_upd ('apply', t, s) adds U_ts and the restriction of the parent's accumulator to the
    leaf in one rounded addition. The leaf tasks ('lu', 'trsl', 'trsu') are the leaf cases of
    Alg 2 and Alg 3 and its mirror.
    """

    def __init__(self, hm, parent, eps=None, rank_cap=None):
        super().__init__(hm, eps, rank_cap)
        self.parent = parent

    def _pulled(self, key):
        own = list(self.acc.get(key, []))
        p = self.parent.get(key)
        if p is None:
            return own
        P, C = self.bt.blocks[p], self.bt.blocks[key]
        ro, co = C.row.lo - P.row.lo, C.col.lo - P.col.lo
        m, n = C.row.size, C.col.size
        for (r0, c0, W, Z) in self.acc.get(p, []):
            ir0, ir1 = max(r0, ro), min(r0 + W.shape[0], ro + m)
            ic0, ic1 = max(c0, co), min(c0 + Z.shape[0], co + n)
            if ir0 < ir1 and ic0 < ic1:
                own.append((ir0 - ro, ic0 - co, W[ir0 - r0:ir1 - r0], Z[ic0 - c0:ic1 - c0]))
        return own

    def run(self, task):
        ty, a, b, c = task
        if ty == "lu":
            self.leaf_lu(self.blk(a, a))
        elif ty == "trsl":
            self.leaf_trsl(self.cl[a], self.blk(a, b))
        elif ty == "trsu":
            self.leaf_trsu(self.cl[a], self.blk(b, a))
        elif ty == "add":
            acc = self.acc.setdefault((a, c), [])
            for (r0, c0, W, Z) in self.product(self.blk(a, b), self.blk(b, c)):
                acc.append((r0, c0, -W, Z))
        elif ty == "shift":
            self.acc[(a, b)] = self._pulled((a, b))
        elif ty == "apply":
            C = self.blk(a, b)
            pieces = self._pulled((a, b))
            if pieces:
                self.apply_to_leaf(C, 1.0, pieces, C.row.lo, C.col.lo)
        else:
            raise ValueError(f"unknown task {task}")

    def run_all(self, order):
        for t in order:
            self.run(t)
        return self


class LowRankAccuHLUFactor(AccuHLUFactor):
    """Accumulator H-LU with accumulators in factorised low-rank form (§2.3 names it the default
    format): U_ts is a matrix U V^T over the whole block (t, s), every addition to it is a
    rounded addition at the factorization's eps (no rank cap: an accumulator of a large block
    may need more than the cap of a leaf), shift_upd adds the restriction of the parent's U V^T
    to the son's accumulator (a rounded addition when the son's is not empty), and apply_upd
    adds the accumulator to the leaf. A dense leaf keeps a dense accumulator (no rounding).

    Counts every rounded addition in ``stats.truncations``.
    """

    def _dense_leaf(self, C):
        return C.is_leaf and isinstance(self.M[C.key], Dense)

    def _add_lr(self, C, U, V):
        """U_C := U_C + U V^T (U, V over the whole block C)."""
        old = self.acc.get(C.key)
        if self._dense_leaf(C):
            self.acc[C.key] = (U @ V.T) if old is None else old + U @ V.T
            return
        if old is not None:
            U, V = np.hstack([old[0], U]), np.hstack([old[1], V])
        cap = min(C.row.size, C.col.size)
        self.acc[C.key] = truncate(U, V, self.eps, cap, self.stats)

    def add_upd(self, alpha, A, B, C):
        if not (A.is_leaf or B.is_leaf or C.is_leaf):
            self.pending.setdefault(C.key, []).append((alpha, A, B))
            return
        m, n = C.row.size, C.col.size
        Ws, Zs = [], []
        for (r0, c0, W, Z) in self.product(A, B):
            Wp = np.zeros((m, W.shape[1]))
            Zp = np.zeros((n, Z.shape[1]))
            Wp[r0:r0 + W.shape[0]] = alpha * W
            Zp[c0:c0 + Z.shape[0]] = Z
            Ws.append(Wp)
            Zs.append(Zp)
        if Ws:
            self._add_lr(C, np.hstack(Ws), np.hstack(Zs))

    def shift_upd(self, C):
        acc = self.acc.pop(C.key, None)
        pend = self.pending.pop(C.key, [])
        for i in range(2):
            for j in range(2):
                Cs = C.sons[i][j]
                if acc is not None:
                    r0, c0 = Cs.row.lo - C.row.lo, Cs.col.lo - C.col.lo
                    self._add_lr(Cs, acc[0][r0:r0 + Cs.row.size], acc[1][c0:c0 + Cs.col.size])
                for (alpha, A, B) in pend:
                    for l in range(2):
                        self.add_upd(alpha, A.sons[i][l], B.sons[l][j], Cs)

    def apply_upd(self, C):
        if not C.is_leaf:
            self.shift_upd(C)
            for i in range(2):
                for j in range(2):
                    self.apply_upd(C.sons[i][j])
            return
        acc = self.acc.pop(C.key, None)
        if acc is None:
            return
        st = self.M[C.key]
        if isinstance(st, Dense):
            st.D += acc
            self.stats.flops += st.D.size
        else:
            self.apply_to_leaf(C, 1.0, [(0, 0, acc[0], acc[1])], C.row.lo, C.col.lo)


class CoarseAccuHLUFactor(AccuHLUFactor):
    """Accumulator H-LU whose accumulators collect pieces without rounding and are compressed
    once, when shift_upd passes them to the sons: the pieces of a structured block (its own
    products and the share of its parent) become one rounded addition over the whole block, so
    each son receives a single low-rank piece from above. A leaf adds its pieces in one rounded
    addition as in the piece-list form. (§2.3 leaves the accumulator format open.)"""

    def shift_upd(self, C):
        acc = self.acc.pop(C.key, [])
        if acc:
            m, n = C.row.size, C.col.size
            Ws, Zs = [], []
            for (r0, c0, Wp, Zp) in acc:
                a = np.zeros((m, Wp.shape[1]))
                a[r0:r0 + Wp.shape[0]] = Wp
                b = np.zeros((n, Zp.shape[1]))
                b[c0:c0 + Zp.shape[0]] = Zp
                Ws.append(a)
                Zs.append(b)
            U, V = truncate(np.hstack(Ws), np.hstack(Zs), self.eps, min(m, n), self.stats)
            self.acc[C.key] = [(0, 0, U, V)]
        super().shift_upd(C)
