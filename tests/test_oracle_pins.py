"""Pins of the FP64 oracle against facts the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: values the paper prints
(Fig. 3, Fig. 4), closed forms, brute force on tiny inputs, independent library routines for
special cases, and invariants.  Plausible mistakes (a dropped term, a transposed operand, a
wrong sign, a skipped pivot) fail at least one of them; ``test_planted_*`` check that.
"""
import math

import numpy as np
import pytest
import scipy.spatial

import hm_workloads as W
from oracle import dag as D
from oracle.geometry import kernel_block, mean_nn_spacing
from oracle.hlu import HLUFactor, hmatrix_matvec
from oracle.hmatrix import HMatrix, LowRank, aca, truncate
from oracle.trees import BlockTree, ClusterTree, admissible
from tests.golden import read_graph_fixture


# ---------------------------------------------------------------- kernel entries, spacing h
def test_kernel_closed_form():
    p = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    h = mean_nn_spacing(p)
    assert h == 1.0
    A = kernel_block(p, p, h)
    assert A[0, 0] == pytest.approx(1.0 / (4 * math.pi * h), rel=1e-15)
    assert A[0, 1] == pytest.approx(1.0 / (4 * math.pi * (1.0 + h)), rel=1e-15)
    assert A[1, 0] == A[0, 1]


def test_mean_nn_spacing_matches_kdtree():
    p = W.fibonacci_sphere(3000, 5)
    d, _ = scipy.spatial.cKDTree(p).query(p, k=2)
    assert mean_nn_spacing(p) == pytest.approx(d[:, 1].mean(), rel=1e-13)


# ---------------------------------------------------------------- cluster tree, block tree
def test_cluster_tree_small_line_by_hand():
    ct = ClusterTree(W.line_points(8), leaf_size=2)
    got = [(c.lo, c.hi) for c in ct.clusters]
    assert got == [(0, 8), (0, 4), (0, 2), (2, 4), (4, 8), (4, 6), (6, 8)]
    assert list(ct.perm) == list(range(8))


@pytest.mark.parametrize("geom,n", [("sphere", 4000), ("cube", 4000)])
def test_cluster_tree_bisection_invariants(geom, n):
    p = W.points_for(geom, n, 3)
    ct = ClusterTree(p, 64)
    assert sorted(ct.perm.tolist()) == list(range(n))
    pp = p[ct.perm]
    for c in ct.clusters:
        pts = pp[c.lo:c.hi]
        assert np.all(pts.min(axis=0) == np.array(c.bmin))
        assert np.all(pts.max(axis=0) == np.array(c.bmax))
        if c.is_leaf:
            assert c.size <= 64
            continue
        assert c.size > 64
        s0, s1 = c.sons
        assert (s0.lo, s1.hi) == (c.lo, c.hi) and s0.hi == s1.lo
        ext = np.array(c.bmax) - np.array(c.bmin)
        axis = int(np.argmax(ext))
        mid = 0.5 * (c.bmin[axis] + c.bmax[axis])
        if np.all(pts[: s0.size, axis] < mid) and np.all(pts[s0.size:, axis] >= mid):
            continue
        # median fallback: son 0 holds the floor(m/2) smallest coordinates
        assert s0.size == c.size // 2
        assert pts[: s0.size, axis].max() <= pts[s0.size:, axis].min()


def test_block_tree_partition_and_admissibility():
    p = W.fibonacci_sphere(2048, 11)
    ct = ClusterTree(p, 64)
    bt = BlockTree(ct, 2.0)
    n = len(p)
    cover = np.zeros((n, n), dtype=np.int32)
    pp = p[ct.perm]
    for b in bt.leaves():
        cover[b.row.lo:b.row.hi, b.col.lo:b.col.hi] += 1
        t, s = pp[b.row.lo:b.row.hi], pp[b.col.lo:b.col.hi]
        dmin = scipy.spatial.distance.cdist(t, s).min()
        if b.adm:
            # box diam >= point diameter and box dist <= point distance, so the
            # admissibility condition must hold for the point sets themselves
            dt = scipy.spatial.distance.pdist(t).max() if len(t) > 1 else 0.0
            ds = scipy.spatial.distance.pdist(s).max() if len(s) > 1 else 0.0
            assert min(dt, ds) <= 2.0 * dmin
            assert dmin > 0
        else:
            assert b.row.is_leaf or b.col.is_leaf
    assert np.all(cover == 1)
    assert any(b.adm for b in bt.leaves())


def test_admissibility_boundary_is_inclusive():
    # two unit segments on a line: diam = 1, dist = 0.5 -> min diam <= 2 dist holds with equality
    p = np.array([[0.0, 0, 0], [1.0, 0, 0], [1.5, 0, 0], [2.5, 0, 0]])
    ct = ClusterTree(p, 2)
    a, b = ct.root.sons
    assert admissible(a, b, 2.0)
    assert not admissible(a, b, 1.999)
    assert not admissible(a, a, 1e9)   # dist = 0 is never admissible


# ---------------------------------------------------------------- task graph (Alg 9-11)
def _dag(points, leaf, eta):
    ct = ClusterTree(points, leaf)
    bt = BlockTree(ct, eta)
    b = D.TaskGraphBuilder(ct, bt)
    nodes, edges = b.compute_dag()
    return b, nodes, edges


def test_fig3_hlu_refinement_exact():
    nodes_g, edges_g, _ = read_graph_fixture("fig3_hlu_refinement.txt")
    _, nodes, edges = _dag(W.line_points(128), 64, 2.0)
    assert sorted(nodes) == sorted(nodes_g)
    assert sorted(edges) == sorted(edges_g)


def test_fig4_inherited_and_local_edges():
    _, _, tagged = read_graph_fixture("fig4_inherited_edges.txt")
    _, nodes, edges = _dag(W.line_points(256), 64, 0.0)
    es = set(edges)
    for kind, a, b in tagged:
        assert (a, b) in es, (kind, a, b)


@pytest.mark.parametrize("nleaf", [2, 4, 8])
def test_tiled_lu_node_count_closed_form(nleaf):
    # eta = 0: nothing admissible; H-LU performs the tiled LU task set
    _, nodes, _ = _dag(W.line_points(64 * nleaf), 64, 0.0)
    N = nleaf
    assert len(nodes) == N + N * (N - 1) + (N - 1) * N * (2 * N - 1) // 6


def _closure(nodes, edges):
    idx = {t: i for i, t in enumerate(nodes)}
    n = len(nodes)
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[idx[a]].append(idx[b])
    reach = []
    for s in range(n):
        seen = np.zeros(n, dtype=bool)
        st = list(adj[s])
        while st:
            v = st.pop()
            if not seen[v]:
                seen[v] = True
                st.extend(adj[v])
        reach.append(seen)
    return idx, np.array(reach)


@pytest.mark.parametrize("geom,n,eta", [("line", 512, 0.0), ("sphere", 1024, 2.0),
                                        ("cube", 1024, 2.0)])
def test_dag_matches_brute_force_dependencies(geom, n, eta):
    """Alg 11's graph has exactly the reachability of all RAW conflicts in sequential order."""
    b, nodes, edges = _dag(W.points_for(geom, n, 7), 64, eta)
    seq = D.sequential_leaf_order(b)
    assert len(seq) == len(set(seq)) == len(nodes)
    assert set(seq) == set(nodes)
    pos = {t: i for i, t in enumerate(seq)}
    for a, c in edges:           # every edge is a forward Def 3.2 dependency
        assert pos[a] < pos[c] and b.precedes(a, c)
    D.levels(nodes, edges)       # acyclic
    idx, reach = _closure(seq, edges)
    for i, ti in enumerate(seq):
        for j in range(i + 1, len(seq)):
            if b.precedes(ti, seq[j]):
                assert reach[i, j], (ti, seq[j])
    # and nothing beyond the transitive closure of true dependencies
    raw = [(seq[i], seq[j]) for i in range(len(seq)) for j in range(i + 1, len(seq))
           if b.precedes(seq[i], seq[j])]
    _, reach_raw = _closure(seq, raw)
    assert np.array_equal(reach, reach_raw)


def test_every_leaf_update_triple_once():
    b, nodes, _ = _dag(W.fibonacci_sphere(2048, 11), 64, 2.0)
    muls = [t for t in nodes if t[0] == D.MUL]
    assert len(muls) == len(set(muls))
    # every (row, col) block is factorized or solved exactly once
    solves = [(t[1], t[2]) if t[0] != D.TRSU else (t[2], t[1]) for t in nodes if t[0] != D.MUL]
    assert len(solves) == len(set(solves))


# ---------------------------------------------------------------- truncation, compression
def _known_svd(m, n, s, seed):
    rng = np.random.default_rng(seed)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, len(s))))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, len(s))))
    return Q1, np.asarray(s), Q2


def test_truncate_closed_form_singular_values():
    Q1, s, Q2 = _known_svd(90, 70, [3.0, 1.0, 2e-2, 1e-6, 1e-9], 0)
    # split the product into a stacked, redundant factor pair
    Wf = np.hstack([Q1 * s, 0.5 * Q1[:, :2] * s[:2]])
    Zf = np.hstack([Q2, -Q2[:, :2]])
    exact = Q1 @ np.diag(s) @ Q2.T - 0.5 * Q1[:, :2] @ np.diag(s[:2]) @ Q2[:, :2].T
    sv = np.array([1.5, 0.5, 2e-2, 1e-6, 1e-9])            # exact singular values
    U, V = truncate(Wf, Zf, 1e-5, 64)
    assert U.shape[1] == 3                                 # 1e-6 < 1e-5 * 1.5
    assert np.linalg.norm(U @ V.T - exact, 2) == pytest.approx(1e-6, rel=1e-6)
    assert np.allclose(V.T @ V, np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.norm(U, axis=0), sv[:3], rtol=1e-12)
    U2, V2 = truncate(Wf, Zf, 1e-5, 2)                     # the rank cap wins
    assert U2.shape[1] == 2
    U0, V0 = truncate(np.zeros((5, 3)), np.ones((4, 3)), 1e-5, 8)
    assert U0.shape == (5, 0) and V0.shape == (4, 0)


def test_aca_then_truncate_reaches_eps():
    p = W.fibonacci_sphere(2048, 11)
    ct = ClusterTree(p, 64)
    bt = BlockTree(ct, 2.0)
    big = max((b for b in bt.leaves() if b.adm), key=lambda b: b.row.size * b.col.size)
    pp = p[ct.perm]
    rows, cols = pp[big.row.lo:big.row.hi], pp[big.col.lo:big.col.hi]
    h = mean_nn_spacing(p)
    Dn = kernel_block(rows, cols, h)
    U0, V0 = aca(rows, cols, h, 1e-7, 200)
    U, V = truncate(U0, V0, 1e-6, 64)
    err = np.linalg.norm(Dn - U @ V.T, 2) / np.linalg.norm(Dn, 2)
    assert err < 3e-6
    s = np.linalg.svd(Dn, compute_uv=False)
    assert U.shape[1] == int(np.count_nonzero(s > 1e-6 * s[0]))


# ---------------------------------------------------------------- H-LU, solve, matvec
def _dense_lu_check(hm, f, tol):
    A = hm.exact_dense()
    X = np.random.default_rng(3).standard_normal((hm.n, 6))
    E = A @ X - f.apply_lu(X)
    return np.linalg.norm(E) / np.linalg.norm(A @ X)


def test_hlu_all_dense_equals_dense_lu_and_solve():
    p = W.fibonacci_sphere(300, 2)
    hm = HMatrix(p, 64, 0.0, 1e-14, 64)
    f = HLUFactor(hm).factor()
    assert _dense_lu_check(hm, f, 0) < 1e-14
    b = np.random.default_rng(4).standard_normal(300)
    x = f.solve(b)
    Ao = kernel_block(p, p, hm.h)
    assert np.linalg.norm(x - np.linalg.solve(Ao, b)) / np.linalg.norm(x) < 1e-12


def _permute_within_leaf_rows(hm, seed):
    """Row-permute the matrix inside every leaf cluster so that partial pivoting must act."""
    rng = np.random.default_rng(seed)
    pi = np.arange(hm.n)
    for c in hm.ct.leaves:
        pi[c.lo:c.hi] = c.lo + rng.permutation(c.size)
    for b in hm.bt.leaves():
        st = hm.store[b.key]
        loc = pi[b.row.lo:b.row.hi] - b.row.lo
        if isinstance(st, LowRank):
            st.U = st.U[loc]
        else:
            st.D = st.D[loc]
    return pi


@pytest.mark.parametrize("eta,eps,tol", [(0.0, 1e-14, 1e-13), (2.0, 1e-12, 1e-10)])
def test_hlu_with_pivoting(eta, eps, tol):
    p = W.cube_surface(700, 9)
    hm = HMatrix(p, 64, eta, eps, 64)
    pi = _permute_within_leaf_rows(hm, 1)
    f = HLUFactor(hm).factor()
    A = hm.exact_dense()[pi]
    X = np.random.default_rng(3).standard_normal((hm.n, 4))
    err = np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X)
    assert err < tol
    b = np.random.default_rng(5).standard_normal(hm.n)
    y = np.linalg.solve(A, b)                    # permuted-order dense solve
    Y = f.lsolve(hm.ct.root, b[:, None])
    Xs = f.usolve(hm.ct.root, Y)[:, 0]
    assert np.linalg.norm(Xs - y) / np.linalg.norm(y) < 1e3 * tol


def test_hlu_accuracy_within_ten_eps():
    p = W.fibonacci_sphere(1024, 11)
    hm = HMatrix(p, 64, 2.0, 1e-4, 64)
    assert any(isinstance(s, LowRank) for s in hm.store.values())
    f = HLUFactor(hm).factor()
    A = hm.exact_dense()
    err = np.linalg.norm(A - f.apply_lu(np.eye(hm.n)), 2) / np.linalg.norm(A, 2)
    assert err <= 10 * 1e-4
    assert f.stats.truncations > 0


def test_hmatrix_matvec_against_exact_kernel():
    p = W.fibonacci_sphere(1024, 11)
    hm = HMatrix(p, 64, 2.0, 1e-8, 64)
    x = np.random.default_rng(1).standard_normal(1024)
    y = hmatrix_matvec(hm, x)
    ye = kernel_block(p, p, hm.h) @ x
    assert np.linalg.norm(y - ye) / np.linalg.norm(ye) < 1e-7


# ---------------------------------------------------------------- planted mistakes are caught
def test_planted_missing_pivots_is_caught(monkeypatch):
    p = W.cube_surface(300, 9)
    hm = HMatrix(p, 64, 0.0, 1e-14, 64)
    pi = _permute_within_leaf_rows(hm, 1)
    orig = HLUFactor.lsolve

    def no_pivot_lsolve(self, t, R):
        b = self.bt.get(t, t)
        if b.is_leaf:
            st = self.M[b.key]
            saved = st.piv
            st.piv = np.arange(len(saved))
            try:
                return orig(self, t, R)
            finally:
                st.piv = saved
        return orig(self, t, R)

    monkeypatch.setattr(HLUFactor, "lsolve", no_pivot_lsolve)
    f = HLUFactor(hm).factor()
    A = hm.exact_dense()[pi]
    X = np.random.default_rng(3).standard_normal((hm.n, 3))
    assert np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X) > 1e-3


def test_planted_sign_error_in_update_is_caught(monkeypatch):
    p = W.fibonacci_sphere(600, 2)
    hm = HMatrix(p, 64, 2.0, 1e-10, 64)
    orig = HLUFactor.hmul
    monkeypatch.setattr(HLUFactor, "hmul", lambda self, a, A, B, C: orig(self, -a, A, B, C))
    f = HLUFactor(hm).factor()
    A = hm.exact_dense()
    X = np.random.default_rng(3).standard_normal((hm.n, 3))
    assert np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X) > 1e-3


def test_planted_transposed_low_rank_solve_is_caught(monkeypatch):
    p = W.fibonacci_sphere(1024, 11)
    hm = HMatrix(p, 64, 2.0, 1e-10, 64)
    monkeypatch.setattr(HLUFactor, "utsolve", lambda self, t, R: self.usolve(t, R))
    f = HLUFactor(hm).factor()
    A = hm.exact_dense()
    X = np.random.default_rng(3).standard_normal((hm.n, 3))
    assert np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X) > 1e-3


def test_sparsification_keeps_reachability_and_levels():
    """Alg 12 removes only edges whose target is reached by another path: the standard graph keeps
    its transitive closure and every longest-path level, with fewer edges (§4.1)."""
    hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, 1e-6, 64)
    n1, e1 = D.TaskGraphBuilder(hm.ct, hm.bt).compute_dag()
    n2, e2 = D.TaskGraphBuilder(hm.ct, hm.bt).compute_dag(sparsify=True)
    assert sorted(n1) == sorted(n2) and set(e2) < set(e1)
    l1, l2 = D.levels(n1, e1), D.levels(n2, e2)
    assert all(l1[t] == l2[t] for t in n1)

    def closure(nodes, edges):
        idx = {t: i for i, t in enumerate(sorted(nodes))}
        out = {t: [] for t in nodes}
        for a, b in edges:
            out[a].append(b)
        reach = {}
        for t in sorted(nodes, key=lambda t: -l1[t]):   # sinks first
            m = 0
            for b in out[t]:
                m |= reach[b] | (1 << idx[b])
            reach[t] = m
        return reach

    assert closure(n1, e1) == closure(n2, e2)


def test_fp32_products_accuracy_and_refinement():
    """Products in FP32 (operands and accumulation), FP64 elsewhere: no visible loss at eps = 1e-4,
    the FP32 floor (~1e-8 relative) showing at eps = 1e-8, and FP64 refinement with these
    factors reaching a residual of 1e-10 in a few steps."""
    from oracle.mixed import MixedHLUFactor, refine
    X = np.random.default_rng(3).standard_normal((1024, 4))
    errs = {}
    for eps in (1e-4, 1e-8):
        hm = HMatrix(W.fibonacci_sphere(1024, 11), 64, 2.0, eps, 64)
        A = hm.exact_dense()
        rel = lambda f: np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X)
        f64, f32 = HLUFactor(hm).factor(), MixedHLUFactor(hm).factor()
        errs[eps] = (rel(f64), rel(f32))
        if eps == 1e-4:
            b = np.random.default_rng(4).standard_normal((1024, 1))
            _, steps, res = refine(A, f32, b, tol=1e-10)
            assert res <= 1e-10 and steps <= 3
    e64, e32 = errs[1e-4]
    assert e32 <= 10 * 1e-4 and abs(e32 - e64) <= 0.05 * e64
    e64, e32 = errs[1e-8]
    assert e32 > 3 * e64 and e32 < 1e-6


def test_wave_parallel_runner_matches_recursion():
    """The task-graph runner (levels of Alg 11 on a thread pool) computes the same factorization
    as the recursion up to the truncations' rounding: same truncation count, both within
    10 eps, and their products within 10 eps of each other."""
    from oracle.wave_parallel import WaveParallelHLU
    p = W.cube_surface(900, 4)
    hm = HMatrix(p, 64, 2.0, 1e-6, 64)
    f1 = HLUFactor(hm).factor()
    f2 = WaveParallelHLU(hm, threads=4).factor()
    assert f2.waves > 1 and f2.tasks > f2.waves
    assert f2.stats.truncations == f1.stats.truncations
    assert abs(f2.stats.flops - f1.stats.flops) <= 1e-6 * f1.stats.flops
    A = hm.exact_dense()
    X = np.random.default_rng(3).standard_normal((hm.n, 4))
    e1 = np.linalg.norm(A @ X - f1.apply_lu(X)) / np.linalg.norm(A @ X)
    e2 = np.linalg.norm(A @ X - f2.apply_lu(X)) / np.linalg.norm(A @ X)
    assert e1 <= 1e-5 and e2 <= 1e-5
    assert np.linalg.norm(f1.apply_lu(X) - f2.apply_lu(X)) / np.linalg.norm(A @ X) <= 1e-5


def test_wave_parallel_runner_needs_the_level_order():
    """Planted mistake: running the levels in reverse order breaks the factorization."""
    from oracle.wave_parallel import WaveParallelHLU
    p = W.cube_surface(600, 4)
    hm = HMatrix(p, 64, 2.0, 1e-6, 64)
    f = WaveParallelHLU(hm, threads=2).plan()
    f._waves = f._waves[::-1]
    try:                      # a task may meet a block in the wrong state and fail outright
        f.factor()
        A = hm.exact_dense()
        X = np.random.default_rng(3).standard_normal((hm.n, 2))
        assert np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X) > 1e-2
    except (AttributeError, TypeError, ValueError, np.linalg.LinAlgError):
        pass
