"""Pins of the accumulator-based H-LU of the oracle (§2.3, Alg 4-8): the same factors as dense LU
when nothing is compressed, the H-LU accuracy bound with compression and pivoting, fewer
truncations than the recursive H-LU (the point of accumulating), and planted mistakes in the
accumulator bookkeeping that the pins catch."""
import numpy as np
import pytest

import hm_workloads as W
from oracle.accu import AccuHLUFactor
from oracle.geometry import kernel_block
from oracle.hlu import HLUFactor
from oracle.hmatrix import HMatrix, LowRank
from oracle.trees import BlockTree, ClusterTree
from tests.test_oracle_pins import _permute_within_leaf_rows


def _rel(A, f, X):
    return np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X)


def test_accumulator_all_dense_equals_dense_lu():
    p = W.fibonacci_sphere(300, 2)
    hm = HMatrix(p, 64, 0.0, 1e-14, 64)
    f = AccuHLUFactor(hm).factor()
    A = hm.exact_dense()
    assert _rel(A, f, np.eye(hm.n)) < 1e-14
    b = np.random.default_rng(4).standard_normal(hm.n)
    x = f.solve(b)
    assert np.linalg.norm(x - np.linalg.solve(kernel_block(p, p, hm.h), b)) / np.linalg.norm(x) < 1e-12
    assert f.stats.truncations == 0


@pytest.mark.parametrize("eta,eps,tol", [(0.0, 1e-14, 1e-13), (2.0, 1e-12, 1e-10)])
def test_accumulator_with_pivoting(eta, eps, tol):
    p = W.cube_surface(700, 9)
    hm = HMatrix(p, 64, eta, eps, 64)
    pi = _permute_within_leaf_rows(hm, 1)
    f = AccuHLUFactor(hm).factor()
    A = hm.exact_dense()[pi]
    assert _rel(A, f, np.random.default_rng(3).standard_normal((hm.n, 4))) < tol


def test_accumulator_within_ten_eps_and_fewer_truncations():
    p = W.fibonacci_sphere(1024, 11)
    hm = HMatrix(p, 64, 2.0, 1e-4, 64)
    assert any(isinstance(s, LowRank) for s in hm.store.values())
    A = hm.exact_dense()
    fa = AccuHLUFactor(hm).factor()
    err = np.linalg.norm(A - fa.apply_lu(np.eye(hm.n)), 2) / np.linalg.norm(A, 2)
    assert err <= 10 * 1e-4
    fs = HLUFactor(hm).factor()
    assert 0 < fa.stats.truncations < fs.stats.truncations


def test_planted_dropped_pending_update_is_caught(monkeypatch):
    p = W.fibonacci_sphere(1024, 11)
    hm = HMatrix(p, 64, 2.0, 1e-10, 64)
    orig = AccuHLUFactor.shift_upd

    def lossy_shift(self, C):
        self.pending.pop(C.key, None)            # forget the deferred products
        orig(self, C)

    monkeypatch.setattr(AccuHLUFactor, "shift_upd", lossy_shift)
    f = AccuHLUFactor(hm).factor()
    assert _rel(hm.exact_dense(), f, np.random.default_rng(3).standard_normal((hm.n, 2))) > 1e-3


def test_planted_misplaced_restriction_is_caught(monkeypatch):
    """Restricting an accumulator to a son with the son's row offset in place of its column offset
    puts the pieces of off-diagonal sons in the wrong columns."""
    p = W.fibonacci_sphere(1024, 11)
    hm = HMatrix(p, 64, 2.0, 1e-10, 64)

    def swapped_shift(self, C):
        acc = self.acc.pop(C.key, [])
        pend = self.pending.pop(C.key, [])
        for i in range(2):
            for j in range(2):
                Cs = C.sons[i][j]
                ro = Cs.row.lo - C.row.lo
                m, n = Cs.row.size, Cs.col.size
                for (r0, c0, Wp, Zp) in acc:
                    ir0, ir1 = max(r0, ro), min(r0 + Wp.shape[0], ro + m)
                    ic0, ic1 = max(c0, ro), min(c0 + Zp.shape[0], ro + n)
                    if ir0 < ir1 and ic0 < ic1:
                        self.acc.setdefault(Cs.key, []).append(
                            (ir0 - ro, ic0 - ro, Wp[ir0 - r0:ir1 - r0], Zp[ic0 - c0:ic1 - c0]))
                for (alpha, A, B) in pend:
                    for l in range(2):
                        self.add_upd(alpha, A.sons[i][l], B.sons[l][j], Cs)

    monkeypatch.setattr(AccuHLUFactor, "shift_upd", swapped_shift)
    f = AccuHLUFactor(hm).factor()
    assert _rel(hm.exact_dense(), f, np.random.default_rng(3).standard_normal((hm.n, 2))) > 1e-3


# -- the task graph of the accumulator H-LU (§3.2, Table 2) -------------------------------------------
import heapq
from collections import defaultdict

from oracle import dag as D
from oracle.accu import AccuTaskRunner


def _graph(hm, builder=D.AccuTaskGraphBuilder):
    b = builder(hm.ct, hm.bt)
    nodes, edges = b.compute_dag()
    return b, nodes, edges


def _level_order(nodes, edges, seed):
    """Waves in level order, shuffled inside each wave (the order the GPU may take)."""
    lev = D.levels(nodes, edges)
    rng = np.random.default_rng(seed)
    return sorted(nodes, key=lambda t: (lev[t], rng.random()))


def _eager_order(nodes, edges, seed):
    """A topological order that runs accumulator tasks as soon as their edges allow."""
    rng = np.random.default_rng(seed)
    indeg, out = defaultdict(int), defaultdict(list)
    for a, b in edges:
        out[a].append(b)
        indeg[b] += 1
    pri = {t: (0 if t[0] in (D.SHIFT, D.APPLY) else 1, rng.random()) for t in nodes}
    heap = [(pri[t], t) for t in nodes if indeg[t] == 0]
    heapq.heapify(heap)
    order = []
    while heap:
        _, t = heapq.heappop(heap)
        order.append(t)
        for s in out[t]:
            indeg[s] -= 1
            if indeg[s] == 0:
                heapq.heappush(heap, (pri[s], s))
    assert len(order) == len(nodes)
    return order


def _ancestors(nodes, edges):
    """Ancestor sets as bit masks over the node index."""
    idx = {t: i for i, t in enumerate(nodes)}
    preds = defaultdict(list)
    for a, b in edges:
        preds[b].append(a)
    anc = {}
    for t in _level_order(nodes, edges, 0):
        m = 0
        for p in preds[t]:
            m |= anc[p] | (1 << idx[p])
        anc[t] = m
    return idx, anc


@pytest.mark.parametrize("geom,n", [("sphere", 1024), ("cube", 700)])
def test_accumulator_graph_tasks(geom, n):
    """The accumulator graph holds the leaf tasks of the standard graph (hmul leaves become
    add_upd leaves), one shift_upd per inner block and one apply_upd per leaf block."""
    hm = HMatrix(W.points_for(geom, n, 21), 64, 2.0, 1e-6, 64)
    _, nodes, edges = _graph(hm)
    std, _ = D.TaskGraphBuilder(hm.ct, hm.bt).compute_dag()
    D.levels(nodes, edges)                       # acyclic
    renamed = sorted((D.ADD,) + t[1:] if t[0] == D.MUL else t for t in std)
    assert sorted(t for t in nodes if t[0] not in (D.SHIFT, D.APPLY)) == renamed
    acc = sorted(t for t in nodes if t[0] in (D.SHIFT, D.APPLY))
    blocks = sorted(((D.APPLY if b.is_leaf else D.SHIFT), b.row.id, b.col.id, -1)
                    for b in hm.bt.blocks.values())
    assert acc == blocks


def test_accumulator_graph_hierarchy_and_updates():
    """Updates reach the leaves top-down (the parent's shift_upd precedes the sons' shift_upd /
    apply_upd), every add_upd into a block precedes the apply_upd of every leaf below it, and
    the apply_upd of a leaf precedes the task that factorises or solves with it."""
    hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, 1e-6, 64)
    b, nodes, edges = _graph(hm)
    idx, anc = _ancestors(nodes, edges)
    acc_task = {(t[1], t[2]): t for t in nodes if t[0] in (D.SHIFT, D.APPLY)}
    for child, par in b.parent.items():
        assert anc[acc_task[child]] >> idx[acc_task[par]] & 1, (par, child)
    for t in nodes:
        if t[0] == D.ADD:
            for leaf in hm.bt.leaves_under(hm.bt.blocks[(t[1], t[3])]):
                assert anc[acc_task[leaf.key]] >> idx[t] & 1, (t, leaf.key)
        elif t[0] in (D.LU, D.TRSL, D.TRSU) and len(nodes) > 1:
            key = (t[2], t[1]) if t[0] == D.TRSU else (t[1], t[2])
            assert anc[t] >> idx[acc_task[key]] & 1, t


@pytest.mark.parametrize("geom,n,eps", [("sphere", 1024, 1e-10), ("cube", 700, 1e-6)])
def test_accumulator_graph_execution_equals_recursion(geom, n, eps):
    """Running the graph's tasks one by one, in level order shuffled inside each level and in an
    order that runs accumulator tasks as early as the edges allow, gives the recursive
    accumulator H-LU (same truncations, same factors up to the order of the stacked pieces)."""
    hm = HMatrix(W.points_for(geom, n, 21), 64, 2.0, eps, 64)
    b, nodes, edges = _graph(hm)
    A = hm.exact_dense()
    X = np.random.default_rng(3).standard_normal((hm.n, 4))
    ref = AccuHLUFactor(hm).factor()
    for order in (_level_order(nodes, edges, 5), _eager_order(nodes, edges, 6)):
        run = AccuTaskRunner(hm, b.parent).run_all(order)
        assert run.stats.truncations == ref.stats.truncations
        assert np.linalg.norm(run.apply_lu(X) - ref.apply_lu(X)) / np.linalg.norm(A @ X) < 100 * eps
        assert _rel(A, run, X) <= 10 * eps


def test_accumulator_graph_literal_and_sparse_readings_have_equal_levels():
    """Table 2 lets add_upd write the global block as well as its accumulator; without that output
    (and with the factorisation and solve tasks reading their own block's accumulator) the graph
    has fewer edges but the same longest-path level for every task: the extra edges are implied."""

    class Sparse(D.AccuTaskGraphBuilder):
        def deps(self, task):
            i, o = super().deps(task)
            ty, a, _, c = task
            if ty == D.ADD:
                o = [self.acc(a, c)]
            elif ty in (D.LU, D.TRSL, D.TRSU):
                i = i + [self.acc(*self._block_of(task))]
            return i, o

    hm = HMatrix(W.fibonacci_sphere(2048, 11), 64, 2.0, 1e-6, 64)
    _, n1, e1 = _graph(hm)
    _, n2, e2 = _graph(hm, Sparse)
    assert sorted(n1) == sorted(n2) and len(e2) < len(e1)
    l1, l2 = D.levels(n1, e1), D.levels(n2, e2)
    assert all(l1[t] == l2[t] for t in n1)


def test_planted_apply_without_parent_accumulator_is_caught(monkeypatch):
    hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, 1e-10, 64)
    orig = D.AccuTaskGraphBuilder.deps

    def deps(self, task):
        i, o = orig(self, task)
        return ([self.acc(task[1], task[2])] if task[0] == D.APPLY else i), o

    monkeypatch.setattr(D.AccuTaskGraphBuilder, "deps", deps)
    b, nodes, edges = _graph(hm)
    run = AccuTaskRunner(hm, b.parent).run_all(_level_order(nodes, edges, 5))
    assert _rel(hm.exact_dense(), run, np.random.default_rng(3).standard_normal((hm.n, 2))) > 1e-3


def test_planted_shift_without_parent_accumulator_is_caught(monkeypatch):
    hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, 1e-6, 64)
    orig = D.AccuTaskGraphBuilder.deps

    def deps(self, task):
        i, o = orig(self, task)
        return ([self.acc(task[1], task[2])] if task[0] == D.SHIFT else i), o

    monkeypatch.setattr(D.AccuTaskGraphBuilder, "deps", deps)
    with pytest.raises(AssertionError):
        test_accumulator_graph_hierarchy_and_updates()


def test_planted_add_without_accumulator_output_is_caught(monkeypatch):
    hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, 1e-10, 64)
    orig = D.AccuTaskGraphBuilder.deps

    def deps(self, task):
        i, o = orig(self, task)
        return i, (o[:1] if task[0] == D.ADD else o)

    monkeypatch.setattr(D.AccuTaskGraphBuilder, "deps", deps)
    b, nodes, edges = _graph(hm)
    run = AccuTaskRunner(hm, b.parent).run_all(_eager_order(nodes, edges, 6))
    assert _rel(hm.exact_dense(), run, np.random.default_rng(3).standard_normal((hm.n, 2))) > 1e-3


# -- the merged accumulator graph (§4.3) ---------------------------------------------------------------
@pytest.mark.parametrize("geom,n,eta", [("sphere", 2048, 2.0), ("cube", 3000, 2.0), ("line", 512, 0.0)])
def test_merged_graph_same_tasks_fewer_edges_same_levels(geom, n, eta):
    """The merged graph has the tasks of the semi-automatic accumulator graph, fewer edges (the
    point of §4.3) and the same longest-path level for every task, so the same waves."""
    hm = HMatrix(W.points_for(geom, n, 21), 64, eta, 1e-6, 64)
    _, n1, e1 = _graph(hm)
    n2, e2 = D.merged_accumulator_dag(hm.ct, hm.bt)
    assert sorted(n1) == sorted(n2) and len(set(e2)) == len(e2) < len(e1)
    l1, l2 = D.levels(n1, e1), D.levels(n2, e2)
    assert all(l1[t] == l2[t] for t in n1)


def test_merged_graph_execution_equals_recursion():
    hm = HMatrix(W.cube_surface(700, 21), 64, 2.0, 1e-6, 64)
    b = D.AccuTaskGraphBuilder(hm.ct, hm.bt)
    nodes, edges = D.merged_accumulator_dag(hm.ct, hm.bt)
    A = hm.exact_dense()
    X = np.random.default_rng(3).standard_normal((hm.n, 4))
    ref = AccuHLUFactor(hm).factor()
    for order in (_level_order(nodes, edges, 7), _eager_order(nodes, edges, 8)):
        run = AccuTaskRunner(hm, b.parent).run_all(order)
        assert run.stats.truncations == ref.stats.truncations
        assert np.linalg.norm(run.apply_lu(X) - ref.apply_lu(X)) / np.linalg.norm(A @ X) < 1e-4
        assert _rel(A, run, X) <= 1e-5


def test_planted_merged_graph_without_add_links_is_caught(monkeypatch):
    """Without the add_upd -> accumulator-task links an eager order applies accumulators early."""
    hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, 1e-10, 64)
    nodes, edges = D.merged_accumulator_dag(hm.ct, hm.bt)
    edges = [(a, b) for a, b in edges if not (a[0] == D.ADD and b[0] in (D.SHIFT, D.APPLY))]
    b = D.AccuTaskGraphBuilder(hm.ct, hm.bt)
    run = AccuTaskRunner(hm, b.parent).run_all(_eager_order(nodes, edges, 6))
    assert _rel(hm.exact_dense(), run, np.random.default_rng(3).standard_normal((hm.n, 2))) > 1e-3


# -- accumulator formats (§2.3 leaves the format open) ---------------------------------------------------
from oracle.accu import CoarseAccuHLUFactor, LowRankAccuHLUFactor


@pytest.mark.parametrize("cls", [LowRankAccuHLUFactor, CoarseAccuHLUFactor])
def test_accumulator_formats_dense_case_and_accuracy(cls):
    p = W.fibonacci_sphere(300, 2)
    hm0 = HMatrix(p, 64, 0.0, 1e-14, 64)
    assert _rel(hm0.exact_dense(), cls(hm0).factor(), np.eye(hm0.n)) < 1e-14
    hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, 1e-4, 64)
    A = hm.exact_dense()
    f = cls(hm).factor()
    assert np.linalg.norm(A - f.apply_lu(np.eye(hm.n)), 2) / np.linalg.norm(A, 2) <= 10 * 1e-4
    assert not f.acc and not f.pending


def test_accumulator_formats_truncation_order():
    """Rounded additions: piece lists (one per low-rank leaf) <= coarse compression (plus one per
    structured block with updates) < low-rank accumulators (one per addition) < recursive H-LU."""
    hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, 1e-6, 64)
    counts = [c(hm).factor().stats.truncations
              for c in (AccuHLUFactor, CoarseAccuHLUFactor, LowRankAccuHLUFactor, HLUFactor)]
    assert counts[0] <= counts[1] < counts[2] < counts[3]


def test_accumulator_edges_of_the_paper_figure():
    """The edges that accumulator handling induces in H-LU, before and after refinement, as the
    figure of §4.1 on sparsification draws them: shift_upd(A_tt) precedes hlu(t0) and
    htrsu(t0, t1) (through shift_upd(A_t1t0) once refined); after refinement shift_upd(A_tt) ->
    shift_upd(A_t0t0) -> hlu(t00) and shift_upd(A_tt) -> shift_upd(A_t1t0) -> the htrsu tasks of
    t00. Two levels below the root, no admissible block (the line, eta = 0)."""
    ct = ClusterTree(W.line_points(256), 64)
    bt = BlockTree(ct, 0.0)
    r = ct.root
    t0, t1 = r.sons
    t00 = t0.sons[0]
    t10, t11 = t1.sons
    nodes, edges = D.AccuTaskGraphBuilder(ct, bt).compute_dag()
    E = set(edges)
    sh = lambda a, b: (D.SHIFT, a.id, b.id, -1)
    assert (sh(r, r), sh(t0, t0)) in E
    assert (sh(t0, t0), (D.LU, t00.id, t00.id, -1)) in E
    assert (sh(r, r), sh(t1, t0)) in E
    assert (sh(t1, t0), (D.TRSU, t00.id, t10.id, -1)) in E
    assert (sh(t1, t0), (D.TRSU, t00.id, t11.id, -1)) in E
    # before refinement: the same dependencies on the unrefined tasks
    b = D.AccuTaskGraphBuilder(ct, bt)
    root = (D.LU, r.id, r.id, -1)
    sub = b.subtasks(root)
    assert sub[0] == sh(r, r)
    assert b.precedes(sub[0], (D.LU, t0.id, t0.id, -1))
    assert b.precedes(sub[0], (D.TRSU, t0.id, t1.id, -1))


def test_sparsification_drops_accumulator_hierarchy():
    """§4.1 warns that removing redundant edges during construction can remove edges the
    accumulator handling needs: with Alg 12 the accumulator graph loses orderings of a parent's
    accumulator task before its sons' (none are lost without it)."""
    hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, 1e-6, 64)

    def misses(sparsify):
        b = D.AccuTaskGraphBuilder(hm.ct, hm.bt)
        nodes, edges = b.compute_dag(sparsify=sparsify)
        idx, anc = _ancestors(nodes, edges)
        acc_task = {(t[1], t[2]): t for t in nodes if t[0] in (D.SHIFT, D.APPLY)}
        return sum(1 for child, par in b.parent.items() if not anc[acc_task[child]] >> idx[acc_task[par]] & 1)

    assert misses(False) == 0
    assert misses(True) > 0
