"""Semi-automatic task-graph construction for H-LU (§3.1: Def 3.1, Def 3.2, Table 1, Alg 9-11).

Oracle; test-only.  Tasks are tuples ``(type, c1, c2, c3)`` of cluster ids:

  ('lu',   t, t, -1)   hlu(A_tt, L_tt, U_tt)                     (Alg 2)
  ('trsl', t, s, -1)   htrsl(L_tt, M_ts, X_ts): L X = M          (Alg 3)
  ('trsu', t, s, -1)   htrsu(U_tt, M_st, X_st): X U = M          (upper mirror of Alg 3)
  ('mul',  t, r, s )   hmul(-1, A_tr, B_rs, C_ts)                (Alg 1)

In H-LU the matrix identifiers are fixed per task type (Table 1 with the arguments of
Alg 2 / Alg 3): hlu reads A and writes L, U; htrsl reads L, A and writes U; htrsu reads
U, A and writes L; hmul reads L, U and writes A.  A data dependency is
(identifier, row cluster, column cluster); two blocks intersect when both their row and
their column index ranges overlap.

Reading of the automatic local edges (Remark on automatic E_t): within the sub-tasks of
one refined task, t_i -> t_j is an edge for i < j in program order whenever Def 3.2 holds.
"""
from __future__ import annotations

from collections import defaultdict, deque

LU, TRSL, TRSU, MUL = "lu", "trsl", "trsu", "mul"
ID_A, ID_L, ID_U = 0, 1, 2


class TaskGraphBuilder:
    def __init__(self, ct, bt):
        self.ct = ct
        self.bt = bt
        self.cl = ct.clusters

    # -- Table 1: input / output data dependencies ---------------------------------------
    def deps(self, task):
        ty, a, b, c = task
        if ty == LU:
            return [(ID_A, a, a)], [(ID_L, a, a), (ID_U, a, a)]
        if ty == TRSL:      # L_aa X_ab = M_ab
            return [(ID_L, a, a), (ID_A, a, b)], [(ID_U, a, b)]
        if ty == TRSU:      # X_ba U_aa = M_ba
            return [(ID_U, a, a), (ID_A, b, a)], [(ID_L, b, a)]
        # MUL: C_ac += A_ab B_bc
        return [(ID_L, a, b), (ID_U, b, c)], [(ID_A, a, c)]

    def _overlap(self, x, y) -> bool:
        cx, cy = self.cl[x], self.cl[y]
        return cx.lo < cy.hi and cy.lo < cx.hi

    def precedes(self, ti, tj) -> bool:
        """Def 3.2: some output of ti and some input of tj share the identifier and intersect."""
        if ti == tj:
            return False
        _, out_i = self.deps(ti)
        in_j, _ = self.deps(tj)
        for (idi, ri, ci) in out_i:
            for (idj, rj, cj) in in_j:
                if idi == idj and self._overlap(ri, rj) and self._overlap(ci, cj):
                    return True
        return False

    # -- refinement: the recursive bodies of Alg 2, Alg 3, its mirror and Alg 1 ----------
    def _leaf(self, r, c) -> bool:
        return self.bt.is_leaf(self.cl[r], self.cl[c])

    def subtasks(self, task) -> list:
        ty, a, b, c = task
        if ty == LU:
            if self._leaf(a, a):
                return []
            t0, t1 = (s.id for s in self.cl[a].sons)
            return [(LU, t0, t0, -1), (TRSU, t0, t1, -1), (TRSL, t0, t1, -1),
                    (MUL, t1, t0, t1), (LU, t1, t1, -1)]
        if ty == TRSL:
            if self._leaf(a, b):
                return []
            t0, t1 = (s.id for s in self.cl[a].sons)
            s0, s1 = (s.id for s in self.cl[b].sons)
            return [(TRSL, t0, s0, -1), (TRSL, t0, s1, -1),
                    (MUL, t1, t0, s0), (MUL, t1, t0, s1),
                    (TRSL, t1, s0, -1), (TRSL, t1, s1, -1)]
        if ty == TRSU:
            if self._leaf(b, a):
                return []
            t0, t1 = (s.id for s in self.cl[a].sons)
            s0, s1 = (s.id for s in self.cl[b].sons)
            return [(TRSU, t0, s0, -1), (TRSU, t0, s1, -1),
                    (MUL, s0, t0, t1), (MUL, s1, t0, t1),
                    (TRSU, t1, s0, -1), (TRSU, t1, s1, -1)]
        # MUL: refine only if none of (a,b), (b,c), (a,c) is a leaf block (Alg 1)
        if self._leaf(a, b) or self._leaf(b, c) or self._leaf(a, c):
            return []
        out = []
        for i in range(2):
            for j in range(2):
                for l in range(2):
                    out.append((MUL, self.cl[a].sons[i].id, self.cl[b].sons[l].id,
                                self.cl[c].sons[j].id))
        return out

    # -- Alg 11 with Alg 9 (refine_sub_deps) and Alg 10 (refine_loc_deps) ---------------
    def compute_dag(self, root_task=None, sparsify=False):
        """Alg 11; with sparsify, every iteration ends with Alg 12 on each task of the work set."""
        if root_task is None:
            r = self.ct.root.id
            root_task = (LU, r, r, -1)
        succ = {root_task: []}          # S_t of every live task
        nodes = []                      # retired tasks: V
        edges = []                      # E
        work = [root_task]              # N
        while work:
            sub = {}
            for g in work:              # generate V_g, E_g
                vg = self.subtasks(g)
                sub[g] = vg
                for i, ti in enumerate(vg):
                    succ[ti] = [tj for tj in vg[i + 1:] if self.precedes(ti, tj)]
            nxt = []
            retire = []
            for g in work:
                vg = sub[g]
                if not vg:
                    old = succ[g]
                    new = []           # refine_loc_deps(g)
                    for x in old:
                        cand = sub.get(x) or [x]
                        for s in cand:
                            if self.precedes(g, s):
                                new.append(s)
                    succ[g] = new
                    if any(sub.get(x) for x in old):
                        nxt.append(g)
                    else:
                        retire.append(g)
                else:
                    for x in succ[g]:  # refine_sub_deps(g)
                        cand = sub.get(x) or [x]
                        for tp in vg:
                            for s in cand:
                                if self.precedes(tp, s):
                                    succ[tp].append(s)
                    nxt.extend(vg)
            if sparsify:
                for g in work:
                    self._sparsify(g, sub, succ)
            for g in retire:
                nodes.append(g)
                edges.extend((g, s) for s in succ[g])
            for g in work:
                if sub[g]:
                    del succ[g]
            work = nxt
        return nodes, edges

    # -- §4.1, Alg 12: removal of redundant edges inside a task's neighbourhood ---------------------
    @staticmethod
    def _sparsify(t, sub, succ):
        """The neighbourhood N is t's sub-tasks (or t) and, for every successor, its sub-tasks (or
        the successor). Every edge (t', s) of t's sub-tasks (or of t) whose target s is also
        reached by a path of length at least two inside N is removed (bfs_2 of Alg 12)."""
        vt = sub[t]
        N = set(vt) if vt else {t}
        for s in succ[t]:
            vs = sub.get(s)
            N.update(vs if vs else (s,))
        for tp in (vt if vt else [t]):
            seen = set()
            stack = []
            for s in succ[tp]:
                if s in N:
                    for u in succ.get(s, ()):
                        if u in N and u not in seen:
                            seen.add(u)
                            stack.append(u)
            while stack:
                v = stack.pop()
                for u in succ.get(v, ()):
                    if u in N and u not in seen:
                        seen.add(u)
                        stack.append(u)
            if seen:
                succ[tp] = [s for s in succ[tp] if s not in seen]


def canonical(nodes, edges):
    """Sorted node list and sorted (src index, dst index) edge list."""
    order = sorted(nodes, key=lambda t: (t[0], t[1], t[2], t[3]))
    index = {t: i for i, t in enumerate(order)}
    e = sorted({(index[a], index[b]) for a, b in edges})
    return order, e


def sequential_leaf_order(builder, root_task=None):
    """Leaf tasks in the order the recursive algorithm executes them (depth-first)."""
    if root_task is None:
        r = builder.ct.root.id
        root_task = (LU, r, r, -1)
    out = []

    def rec(t):
        v = builder.subtasks(t)
        if not v:
            out.append(t)
        for s in v:
            rec(s)

    rec(root_task)
    return out


def levels(nodes, edges):
    """Longest-path level of each node (sources at level 0); raises if the graph has a cycle."""
    indeg = defaultdict(int)
    out = defaultdict(list)
    for a, b in edges:
        out[a].append(b)
        indeg[b] += 1
    lev = {t: 0 for t in nodes}
    q = deque(t for t in nodes if indeg[t] == 0)
    seen = 0
    while q:
        t = q.popleft()
        seen += 1
        for s in out[t]:
            lev[s] = max(lev[s], lev[t] + 1)
            indeg[s] -= 1
            if indeg[s] == 0:
                q.append(s)
    if seen != len(nodes):
        raise ValueError("task graph has a cycle")
    return lev


# -- §3.2: the task graph of the accumulator-based H-LU (Table 2, Alg 7, Alg 8) --------------------
ADD, SHIFT, APPLY = "add", "shift", "apply"


class AccuTaskGraphBuilder(TaskGraphBuilder):
    """Tasks of the accumulator-based H-LU with the data dependencies of Table 2.

    Task tuples: ('lu', t, t, -1), ('trsl', t, s, -1) and ('trsu', t, s, -1) as above;
    ('add', t, r, s) for add_upd(-1, L_tr, U_rs, A_ts) (refined like hmul, Alg 1);
    ('shift', t, s, -1) for shift_upd of the block (t, s); ('apply', t, s, -1) for apply_upd of
    the leaf (t, s).  Every accumulator is a matrix of its own: its identifier is
    ('acc', t, s), so only dependencies on the same block's accumulator can intersect.

    Readings:
    * the parent accumulator a task reads (Table 2) is the accumulator of the parent block in the
      block tree, restricted to the task's own block; the root block has none;
    * shift_upd and apply_upd appear where Alg 7 / Alg 8 call them: a refined hlu / htrsl /
      htrsu starts with shift_upd of its block, and every sub-task of those types whose block is
      a leaf is preceded by apply_upd of that leaf in the sub-task list;
    * add_upd of three structured blocks refines into the eight products of the sons (what
      shift_upd does with a pending product), so leaf add_upd tasks are formed exactly where
      hmul has leaf tasks.
    """

    def __init__(self, ct, bt):
        super().__init__(ct, bt)
        self.parent = {}
        for b in bt.blocks.values():
            for row in b.sons:
                for s in row:
                    self.parent[s.key] = b.key

    @staticmethod
    def acc(r, c):
        return (("acc", r, c), r, c)

    def acc_parent(self, r, c):
        p = self.parent.get((r, c))
        return [] if p is None else [(("acc",) + p, r, c)]

    def deps(self, task):
        ty, a, b, c = task
        if ty == LU:
            return [(ID_A, a, a)] + self.acc_parent(a, a), [(ID_L, a, a), (ID_U, a, a)]
        if ty == TRSL:
            return [(ID_L, a, a), (ID_A, a, b)] + self.acc_parent(a, b), [(ID_U, a, b)]
        if ty == TRSU:
            return [(ID_U, a, a), (ID_A, b, a)] + self.acc_parent(b, a), [(ID_L, b, a)]
        if ty == ADD:
            return [(ID_L, a, b), (ID_U, b, c)], [(ID_A, a, c), self.acc(a, c)]
        if ty == SHIFT:
            return self.acc_parent(a, b) + [self.acc(a, b)], [self.acc(a, b)]
        # APPLY
        return self.acc_parent(a, b) + [self.acc(a, b)], [(ID_A, a, b)]

    def _block_of(self, task):
        ty, a, b, _ = task
        return (b, a) if ty == TRSU else (a, b)

    def subtasks(self, task):
        ty, a, b, c = task
        if ty in (SHIFT, APPLY):
            return []
        if ty == ADD:
            return [(ADD,) + t[1:] for t in super().subtasks((MUL, a, b, c))]
        sub = super().subtasks(task)
        if not sub:
            return []
        out = [(SHIFT,) + self._block_of(task) + (-1,)]
        for t in sub:
            if t[0] == MUL:
                out.append((ADD,) + t[1:])
                continue
            r, s = self._block_of(t)
            if self._leaf(r, s):
                out.append((APPLY, r, s, -1))
            out.append(t)
        return out


def merged_accumulator_dag(ct, bt):
    """The accumulator task graph built in two parts and linked explicitly (§4.3).

    First the accumulator handling alone: one shift_upd per inner block and one apply_upd per
    leaf block, with an edge from the task of every block to the tasks of its sons (the parent's
    accumulator is complete before a son takes its share). Then the standard H-LU graph (Alg 11
    with Table 1; hmul tasks become add_upd), to which two kinds of edges are added: from every
    add_upd to the accumulator task of its destination block, and from the apply_upd of a leaf to
    the task that factorises or solves with that leaf.
    """
    nodes, edges = TaskGraphBuilder(ct, bt).compute_dag()
    ren = {t: ((ADD,) + t[1:] if t[0] == MUL else t) for t in nodes}
    acc = {key: ((SHIFT if b.sons else APPLY), key[0], key[1], -1) for key, b in bt.blocks.items()}
    out_nodes = [ren[t] for t in nodes] + list(acc.values())
    out_edges = [(ren[a], ren[b]) for a, b in edges]
    for key, b in bt.blocks.items():
        for row in b.sons:
            for s in row:
                out_edges.append((acc[key], acc[s.key]))
    for t in out_nodes:
        ty, a, b, c = t
        if ty == ADD:
            out_edges.append((t, acc[(a, c)]))
        elif ty in (LU, TRSL, TRSU):
            out_edges.append((acc[(b, a) if ty == TRSU else (a, b)], t))
    return out_nodes, out_edges
