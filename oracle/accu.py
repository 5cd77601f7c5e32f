"""Accumulator-based H-LU (§2.3: Alg 4 add_upd, Alg 5 apply_upd, Alg 6 shift_upd, Alg 7 hlu and
Alg 8 htrsl with accumulators, and the upper mirror of Alg 8). Oracle; test-only.

Updates are not applied where they arise: add_upd collects the product alpha A B in the
accumulator U_{t,s} of the destination block when one of the three blocks is a leaf (the
product can then be formed), and otherwise records the triple in the pending set P_{t,s}.
Before a block is factorised or solved with, its accumulated updates are shifted down to the
sub-blocks (shift_upd) at each recursive step, and a leaf adds its accumulator once
(apply_upd) before the dense factorisation or solve.

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

from .hlu import HLUFactor


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
