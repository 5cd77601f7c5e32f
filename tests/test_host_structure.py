"""Host logic of the CUDA library against the oracle, bit for bit (CPU only).

The library's cluster tree, block tree and Alg 11 task graph are plain host C++; they must
equal the oracle's exactly (same permutation, same clusters, same leaves and admissibility
decisions, same task set, same edge set) on the seeded workloads, and the library must load
and export every function the public header declares.
"""
import ctypes

import numpy as np
import pytest

import hm_workloads as W
import paper_1911_07531_gb300 as hm
from oracle import dag as D
from oracle.trees import BlockTree, ClusterTree

TYPES = {0: D.LU, 1: D.MUL, 2: D.TRSL, 3: D.TRSU}


@pytest.fixture(scope="module")
def lib():
    hm.build_library()
    return hm.load_library()


def test_library_exports_every_header_symbol(lib):
    names = hm.header_functions()
    assert "hm_lu" in names and "hm_build" in names and "hm_solve" in names and "hm_matvec" in names
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def _compare(points, leaf, eta, check_dag=True):
    S = hm.hm_structure_build(points, leaf, eta).export()
    ct = ClusterTree(points, leaf)
    bt = BlockTree(ct, eta)
    assert np.array_equal(S["perm"], ct.perm)
    got = [tuple(r) for r in S["clusters"][:, :4].tolist()]
    ref = [(c.lo, c.hi, c.sons[0].id if c.sons else -1, c.sons[1].id if c.sons else -1) for c in ct.clusters]
    assert got == ref
    lv = {(r, c): a for r, c, a in S["leaves"].tolist()}
    assert lv == {b.key: int(b.adm) for b in bt.leaves()}
    if not check_dag:
        return S
    b = D.TaskGraphBuilder(ct, bt)
    nodes, edges = b.compute_dag()
    tasks = [(TYPES[t[0]], t[1], t[2], t[3]) for t in S["tasks"].tolist()]
    assert sorted(tasks) == sorted(nodes)
    e_lib = {(tasks[s], tasks[d]) for s, d in S["edges"].tolist()}
    assert len(e_lib) == len(S["edges"])
    assert e_lib == set(edges)
    lev = D.levels(nodes, edges)
    assert all(lev[t] == S["levels"][i] for i, t in enumerate(tasks))
    return S


@pytest.mark.parametrize("geom,n,eta", [("line", 512, 0.0), ("line", 128, 2.0), ("sphere", 2048, 2.0),
                                        ("cube", 3000, 2.0), ("ellipsoid", 1500, 2.0)])
def test_structure_bit_exact_with_oracle(lib, geom, n, eta):
    _compare(W.points_for(geom, n, 21), 64, eta)


def test_structure_trees_bit_exact_larger(lib):
    # trees and admissibility only (the oracle's task graph is slow in Python at this size)
    _compare(W.cube_surface(32768, 31), 64, 2.0, check_dag=False)


def test_structure_degenerate_inputs(lib):
    S = hm.hm_structure_build(np.zeros((1, 3)), 64, 2.0).export()
    assert S["tasks"].tolist() == [[0, 0, 0, -1]] and len(S["edges"]) == 0
    # coincident points force the median split
    p = np.zeros((300, 3))
    _compare(p, 64, 2.0)
    with pytest.raises(hm.HMError):
        hm.hm_structure_build(np.zeros((10, 3)), 0, 2.0)


ACC_TYPES = {0: D.LU, 1: D.ADD, 2: D.TRSL, 3: D.TRSU, 4: D.SHIFT, 5: D.APPLY}


@pytest.mark.parametrize("geom,n,eta", [("line", 512, 0.0), ("sphere", 2048, 2.0), ("cube", 3000, 2.0),
                                        ("ellipsoid", 1500, 2.0)])
@pytest.mark.parametrize("merged", [False, True])
def test_accumulator_graph_bit_exact_with_oracle(lib, geom, n, eta, merged):
    """The library's accumulator task graphs (§3.2 with Table 2; the merged graph of §4.3) equal
    the oracle's: tasks, edges, levels."""
    points = W.points_for(geom, n, 21)
    S = hm.hm_structure_build_accumulator(points, 64, eta, merged).export()
    ct = ClusterTree(points, 64)
    bt = BlockTree(ct, eta)
    if merged:
        nodes, edges = D.merged_accumulator_dag(ct, bt)
    else:
        nodes, edges = D.AccuTaskGraphBuilder(ct, bt).compute_dag()
    tasks = [(ACC_TYPES[t[0]], t[1], t[2], t[3]) for t in S["tasks"].tolist()]
    assert sorted(tasks) == sorted(nodes)
    e_lib = {(tasks[s], tasks[d]) for s, d in S["edges"].tolist()}
    assert len(e_lib) == len(S["edges"])
    assert e_lib == set(edges)
    lev = D.levels(nodes, edges)
    assert all(lev[t] == S["levels"][i] for i, t in enumerate(tasks))


def test_accumulator_graph_single_leaf(lib):
    S = hm.hm_structure_build_accumulator(np.zeros((1, 3)), 64, 2.0).export()
    assert S["tasks"].tolist() == [[0, 0, 0, -1]] and len(S["edges"]) == 0
    S = hm.hm_structure_build_accumulator(np.zeros((1, 3)), 64, 2.0, merged=True).export()
    assert S["tasks"].tolist() == [[0, 0, 0, -1], [5, 0, 0, -1]] and S["edges"].tolist() == [[1, 0]]
    with pytest.raises(hm.HMError):
        hm.hm_structure_build_accumulator(np.zeros((10, 3)), 65, 2.0)


def test_plan_builds_on_host(lib):
    S = hm.hm_structure_build(W.fibonacci_sphere(4096, 11), 64, 2.0, with_plan=True)
    i = S.info
    assert i["plan_launches"] > 0 and i["plan_phases"] >= i["nlevels"]
    assert i["plan_truncations"] > 0 and i["plan_scratch_bytes"] > 0


def test_plan_export_errors(lib):
    S = hm.hm_structure_build(W.fibonacci_sphere(512, 3), 64, 2.0)
    for args in ((10, 1e-6, 64, 1), (0, 0.0, 64, 1), (8, 0.0, 64, 1), (0, 1e-6, 65, 1), (1, 0.0, 64, 0)):
        with pytest.raises(hm.HMError):
            S.plan(*args)
    acc = hm.hm_structure_build_accumulator(W.fibonacci_sphere(512, 3), 64, 2.0)
    with pytest.raises(hm.HMError):
        acc.plan(0, 1e-6, 64)
    P = S.plan(0, 1e-6, 64)
    assert P["sizes"]["nwaves"] == S.info["nlevels"] and len(P["leaves"]) == S.info["nleaves"]
    k = P["launches"]["kind"]
    assert set(k.tolist()) <= set(range(6)) and (P["launches"]["count"] > 0).all()


def test_parallel_planner_equals_sequential(lib):
    """Ranges of waves planned on several host threads and concatenated give the sequential plan
    byte for byte (launch list, every micro-op table, sizes), with and without the wave overlap
    (whose leaf-event analysis also runs on the host threads)."""
    S = hm.hm_structure_build(W.fibonacci_sphere(8192, 21), 64, 2.0)
    for which in (0, 7):
        ref = S.plan(which, 1e-6, 64, threads=1)
        assert ref["sizes"]["nwaves"] >= 64
        for t in (3, 8):
            P = S.plan(which, 1e-6, 64, threads=t)
            for name in ("launches", "getrf", "trsm", "gemm", "copy", "trunc", "entries", "leaves"):
                assert P[name].tobytes() == ref[name].tobytes(), (which, t, name)
            assert P["sizes"].tobytes() == ref["sizes"].tobytes()


def test_parallel_task_graph_equals_serial(lib):
    """The parallel loops of Alg 13 give the serial construction's graph: same task order, same
    edge order, same levels, for the standard and both accumulator graphs (sizes at which the
    work lists are split across threads)."""
    pts = W.fibonacci_sphere(8192, 21)
    builds = (lambda: hm.hm_structure_build(pts, 64, 2.0),
              lambda: hm.hm_structure_build_accumulator(pts, 64, 2.0),
              lambda: hm.hm_structure_build_accumulator(pts, 64, 2.0, merged=True))
    try:
        for make in builds:
            hm.hm_set_host_threads(1)
            ref = make().export()
            for t in (3, 8):
                hm.hm_set_host_threads(t)
                got = make().export()
                for name in ("tasks", "edges", "levels"):
                    assert np.array_equal(got[name], ref[name]), (t, name)
    finally:
        hm.hm_set_host_threads(0)
    with pytest.raises(hm.HMError):
        hm.hm_set_host_threads(-1)


def test_parallel_task_graph_bit_exact_with_oracle_at_8192(lib):
    _compare(W.fibonacci_sphere(8192, 21), 64, 2.0)


def test_lu_batch_rejects_bad_arguments_without_a_device(lib):
    """hm_lu_batch validates its arguments before touching the device."""
    outs = (ctypes.c_void_p * 1)()
    assert lib.hm_lu_batch(None, None, 1, None, outs) == -1
    assert lib.hm_lu_batch(None, (ctypes.c_void_p * 1)(), 0, None, outs) == -1


@pytest.mark.parametrize("accumulators", [False, True])
@pytest.mark.parametrize("geom,n,eta", [("sphere", 2048, 2.0), ("cube", 3000, 2.0), ("line", 512, 0.0)])
def test_sparsified_graph_bit_exact_with_oracle(lib, geom, n, eta, accumulators):
    """Alg 12 (§4.1) during construction: the library's graph equals the oracle's, edge for edge."""
    points = W.points_for(geom, n, 21)
    S = hm.hm_structure_build_sparsified(points, 64, eta, accumulators).export()
    ct = ClusterTree(points, 64)
    bt = BlockTree(ct, eta)
    builder = D.AccuTaskGraphBuilder(ct, bt) if accumulators else D.TaskGraphBuilder(ct, bt)
    nodes, edges = builder.compute_dag(sparsify=True)
    names = ACC_TYPES if accumulators else TYPES
    tasks = [(names[t[0]], t[1], t[2], t[3]) for t in S["tasks"].tolist()]
    assert sorted(tasks) == sorted(nodes)
    assert {(tasks[s], tasks[d]) for s, d in S["edges"].tolist()} == set(edges)
    assert len(S["edges"]) == len(edges)


def test_batching_workload_recipe():
    inst = W.ellipsoid_instances(64)
    ns = np.array([n for n, _ in inst])
    assert len(inst) == 64 and ns.min() >= 4096 and ns.max() <= 65536
    assert 0.3 < np.mean(np.log(ns) < np.log(4096 * 4)) < 0.7      # log-uniform: half below the log-midpoint
    for n, p in inst[:4]:
        assert p.shape == (n, 3) and np.isfinite(p).all()
        r = np.sqrt(((p / np.abs(p).max(axis=0)) ** 2).sum(axis=1))
        assert r.min() > 0.3
    again = W.ellipsoid_instances(64)
    assert all(np.array_equal(a[1], b[1]) for a, b in zip(inst[:3], again[:3]))


def test_no_cpu_fallback_without_a_device(lib):
    """Without a CUDA device the computing path refuses to start (HM_ECUDA): there is no CPU
    fallback behind the boundary."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p()
    assert lib.hm_ctx_create(0, None, hm.ALLOC_FN(), hm.FREE_FN(), None, ctypes.byref(h)) == -3
    assert h.value is None
    assert b"no CUDA device" in lib.hm_last_error()


def test_gemm_split_tuning_changes_the_plan_not_its_operations():
    """The GEMM split target is a process-wide tuning value: a larger FMAs-per-CTA target gives
    GEMM micro-ops no larger splits and the same operations; out-of-range values are refused."""
    import paper_1911_07531_gb300 as hm
    p = W.points_for("cube", 3000, 4)
    S = hm.hm_structure_build(p, 64, 2.0)
    before = hm.hm_get_gemm_work()
    try:
        with pytest.raises(hm.HMError):
            hm.hm_set_gemm_work(0.0)
        hm.hm_set_gemm_work(4096.0)
        g_small = S.plan(0, 1e-6, 64, 1, 1)["gemm"].copy()
        hm.hm_set_gemm_work(262144.0)
        g_large = S.plan(0, 1e-6, 64, 1, 1)["gemm"].copy()
    finally:
        hm.hm_set_gemm_work(before)
    assert len(g_small) == len(g_large)
    sp = lambda g: (g["split"] & 0xffff) * np.maximum(1, g["split"] >> 16)
    assert sp(g_large).sum() < sp(g_small).sum()
    key = lambda g: np.sort(g[["A", "B", "C", "m", "n", "k"]], order=["A", "B", "C", "m", "n", "k"])
    assert (key(g_small) == key(g_large)).all()
