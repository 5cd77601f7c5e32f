"""The library's host plans executed micro-op by micro-op on the CPU (``tests/plan_sim.py``).

The H-LU plan, run on the oracle's H-matrix, must give factors that reproduce A within the
H-LU bound, and the solve plan, run on those factors, must equal the oracle's block
substitution with the same factors: this checks the planner's addresses, strides, dynamic
sizes, phase order and stacking on the host, independently of the CUDA kernels.
"""
import numpy as np
import pytest

import hm_workloads as W
import paper_1911_07531_gb300 as hm
from oracle.hlu import HLUFactor
from oracle.hmatrix import DiagLU, Dense, HMatrix, LowRank
from tests.plan_sim import IS_PIV, IS_RANK, IS_S, SP_F, SP_X, PlanSim


def ref(space, off):
    return ((space + 1) << 60) | int(off)


@pytest.fixture(scope="module")
def lib():
    hm.build_library()
    return hm.load_library()


def _load(sim, leaves, store):
    for lf in leaves:
        st = store[(int(lf["row"]), int(lf["col"]))]
        m, n = int(lf["m"]), int(lf["n"])
        if lf["lr"]:
            k = st.U.shape[1]
            assert k <= int(lf["cap"])
            sim.mat(ref(SP_F, lf["off"]), 1, m, m, k)[:] = st.U
            sim.mat(ref(SP_F, lf["voff"]), 1, n, n, k)[:] = st.V
            sim.i[IS_RANK][int(lf["rank_idx"])] = k
        else:
            sim.mat(ref(SP_F, lf["off"]), 1, m, m, n)[:] = st.D


def _factor(hmat, sim, leaves):
    """The simulated factors in the oracle's factor container."""
    f = HLUFactor(hmat)
    for lf in leaves:
        key = (int(lf["row"]), int(lf["col"]))
        m, n = int(lf["m"]), int(lf["n"])
        if lf["lr"]:
            k = int(sim.i[IS_RANK][int(lf["rank_idx"])])
            U = np.array(sim.mat(ref(SP_F, lf["off"]), 1, m, m, k))
            V = np.array(sim.mat(ref(SP_F, lf["voff"]), 1, n, n, k))
            f.M[key] = LowRank(U, V)
        elif key[0] == key[1]:
            p0 = int(lf["piv_off"])
            f.M[key] = DiagLU(np.array(sim.mat(ref(SP_F, lf["off"]), 1, m, m, n)), sim.i[IS_PIV][p0:p0 + m].copy())
        else:
            f.M[key] = Dense(np.array(sim.mat(ref(SP_F, lf["off"]), 1, m, m, n)))
    return f


@pytest.mark.parametrize("geom,n,eta,eps", [("sphere", 1024, 2.0, 1e-6), ("cube", 1500, 2.0, 1e-4),
                                            ("line", 700, 0.0, 1e-10), ("ellipsoid", 1200, 2.0, 1e-6)])
def test_lu_and_solve_plans_on_the_host(lib, geom, n, eta, eps):
    pts = W.points_for(geom, n, 21)
    hmat = HMatrix(pts, 64, eta, eps, 64)
    S = hm.hm_structure_build(pts, 64, eta)
    P = S.plan(0, eps, 64)
    if geom == "cube":   # stacks beyond one round here: some are rounded as trees (TF_NOSELF sums)
        assert (P["trunc"]["flags"] & 1).any()
    sim = PlanSim(P["sizes"])
    _load(sim, P["leaves"], hmat.store)
    sim.run(P)
    assert sim.singular == 0
    f = _factor(hmat, sim, P["leaves"])
    A = hmat.exact_dense()
    X = np.random.default_rng(3).standard_normal((n, 4))
    err = np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X)
    assert err <= 10 * eps, err
    ref_f = HLUFactor(hmat).factor()
    assert np.linalg.norm(A @ X - ref_f.apply_lu(X)) / np.linalg.norm(A @ X) <= 10 * eps

    # the solve plan on the simulated factors equals the oracle's substitution with them
    nrhs_max = 3
    Q = S.plan(1, 0.0, 64, nrhs_max)
    sol = PlanSim(Q["sizes"], nrhs_space=n * nrhs_max)
    sol.d[SP_F], sol.i[IS_RANK], sol.i[IS_PIV] = sim.d[SP_F], sim.i[IS_RANK], sim.i[IS_PIV]
    B = np.random.default_rng(4).standard_normal((n, 2))
    sol.mat(ref(SP_X, 0), 1, n, n, 2)[:] = B
    sol.i[IS_S][0] = 2
    sol.run(Q)
    Xs = np.array(sol.mat(ref(SP_X, 0), 1, n, n, 2))
    Xo = f.usolve(hmat.ct.root, f.lsolve(hmat.ct.root, B))
    assert np.linalg.norm(Xs - Xo) / np.linalg.norm(Xo) < 1e-12
    assert np.linalg.norm(f.apply_lu(Xs) - B) / np.linalg.norm(B) < 1e-12


def test_plan_sim_catches_a_planted_stride_error(lib):
    """A planner address mistake (here the leading dimension of the low-rank V factors in the
    rebuild products, planted in the exported plan) makes the host run fail its bound."""
    pts = W.fibonacci_sphere(1024, 21)
    hmat = HMatrix(pts, 64, 2.0, 1e-6, 64)
    P = hm.hm_structure_build(pts, 64, 2.0).plan(0, 1e-6, 64)
    sim = PlanSim(P["sizes"])
    _load(sim, P["leaves"], hmat.store)
    core_V = set(int(v) for v in P["trunc"]["V"])
    g = P["gemm"]
    hit = np.array([int(c) in core_V for c in g["C"]])
    assert hit.any()
    g["c_cs"][hit] += 1
    try:
        sim.run(P)
    except AssertionError:
        return
    f = _factor(hmat, sim, P["leaves"])
    A = hmat.exact_dense()
    X = np.random.default_rng(3).standard_normal((hmat.n, 2))
    assert np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X) > 1e-3


@pytest.mark.parametrize("name,pts,eta,eps,cap", [
    ("ragged n = 65", W.fibonacci_sphere(65, 2), 2.0, 1e-6, 64),
    ("all dense", W.fibonacci_sphere(1000, 3), 0.0, 1e-6, 64),
    ("rank cap 4", W.cube_surface(1500, 3), 2.0, 1e-8, 4),
])
def test_lu_plan_edge_cases_on_the_host(lib, name, pts, eta, eps, cap):
    """Ragged leaves, no low-rank block at all, and a rank cap that binds (the plan's rounded
    additions hit the cap exactly as often as the oracle's and end at the same error)."""
    n = len(pts)
    hmat = HMatrix(pts, 64, eta, eps, cap)
    P = hm.hm_structure_build(pts, 64, eta).plan(0, eps, cap)
    sim = PlanSim(P["sizes"])
    _load(sim, P["leaves"], hmat.store)
    sim.run(P)
    f = _factor(hmat, sim, P["leaves"])
    ref_f = HLUFactor(hmat).factor()
    A = hmat.exact_dense()
    X = np.random.default_rng(3).standard_normal((n, 2))
    e_plan = np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X)
    e_ref = np.linalg.norm(A @ X - ref_f.apply_lu(X)) / np.linalg.norm(A @ X)
    if cap < 64:
        assert sim.cap_hits == ref_f.stats.cap_hits > 0
        assert abs(e_plan - e_ref) <= 1e-3 * e_ref
    else:
        assert e_plan <= 10 * eps and sim.cap_hits == 0


def test_matvec_plans_on_the_host(lib):
    """hm_matvec's plans: A x equals the oracle's H-matrix product; U x, then P L of it, equals
    the P L U x of the factors; the fused P L U plan gives the same."""
    from oracle.hlu import hmatrix_matvec
    pts = W.cube_surface(1200, 5)
    n, eps, nr = len(pts), 1e-6, 2
    hmat = HMatrix(pts, 64, 2.0, eps, 64)
    S = hm.hm_structure_build(pts, 64, 2.0)
    P = S.plan(0, eps, 64)
    fac = PlanSim(P["sizes"])
    _load(fac, P["leaves"], hmat.store)
    fac.run(P)
    f = _factor(hmat, fac, P["leaves"])
    x = np.random.default_rng(8).standard_normal((n, nr))

    def run(op, xin):
        Q = S.plan(2 + op, 0.0, 64, nr)
        sim = PlanSim(Q["sizes"], nrhs_space=4 * n * nr)
        sim.d[SP_F], sim.i[IS_RANK], sim.i[IS_PIV] = fac.d[SP_F], fac.i[IS_RANK], fac.i[IS_PIV]
        if op == 0:
            sim.d[3] = np.zeros(int(P["sizes"]["nvalues"]))
            sim.i[3] = np.zeros(int(P["sizes"]["nranks"]), np.int64)
            _load(_Spaces(sim, 3), P["leaves"], hmat.store)
        sim.mat(ref(SP_X, 0), 1, n, n, nr)[:] = xin
        sim.i[IS_S][0] = nr
        sim.run(Q)
        return np.array(sim.mat(ref(SP_X, n * nr), 1, n, n, nr))

    y = run(0, x)
    perm = hmat.ct.perm
    x_orig = np.empty_like(x)
    x_orig[perm] = x
    yo = hmatrix_matvec(hmat, x_orig).reshape(n, nr)[perm]
    assert np.linalg.norm(y - yo) / np.linalg.norm(yo) < 1e-13
    A = hmat.exact_dense()
    assert np.linalg.norm(y - A @ x) / np.linalg.norm(A @ x) < 10 * eps
    plu = f.apply_lu(x)
    assert np.linalg.norm(run(1, run(2, x)) - plu) / np.linalg.norm(plu) < 1e-13
    assert np.linalg.norm(run(3, x) - plu) / np.linalg.norm(plu) < 1e-13


class _Spaces:
    """Loads a leaf table into the matrix-value spaces (3) of a simulator."""

    def __init__(self, sim, space):
        self.sim, self.space = sim, space
        self.i = {IS_RANK: sim.i[space]}

    def mat(self, r, rs, cs, m, n):
        return self.sim.mat(ref(self.space, int(r) & ((1 << 60) - 1)), rs, cs, m, n)


def test_batched_lu_plan_on_the_host(lib):
    """Three independent instances planned as one launch sequence (their waves share phases):
    fewer launches than the three plans together, and every instance's factors equal its own
    plan's result (up to the order of accumulations) and reproduce its matrix within 10 eps."""
    cases = [("sphere", 1024, 11), ("cube", 1500, 3), ("ellipsoid", 700, 4)]
    eps = 1e-6
    hms = [HMatrix(W.points_for(g, n, sd), 64, 2.0, eps, 64) for g, n, sd in cases]
    Ss = [hm.hm_structure_build(W.points_for(g, n, sd), 64, 2.0) for g, n, sd in cases]
    single = [S.plan(0, eps, 64) for S in Ss]
    try:   # the batched planner splits ranges of waves across host threads: same plan
        hm.hm_set_host_threads(1)
        B1 = hm.hm_structure_plan_lu_batch(Ss, eps, 64)
        hm.hm_set_host_threads(6)
        B = hm.hm_structure_plan_lu_batch(Ss, eps, 64)
    finally:
        hm.hm_set_host_threads(0)
    for name in ("launches", "gemm", "trunc", "entries", "copy", "trsm", "getrf", "leaves", "instances"):
        assert B[name].tobytes() == B1[name].tobytes(), name
    assert len(B["launches"]) < sum(len(p["launches"]) for p in single)
    assert len(B["launches"]) >= max(len(p["launches"]) for p in single)
    assert B["sizes"]["nwaves"] == max(p["sizes"]["nwaves"] for p in single)
    assert B["sizes"]["ntrunc"] == sum(p["sizes"]["ntrunc"] for p in single)
    sim = PlanSim(B["sizes"])
    for hmat, I in zip(hms, B["instances"]):
        _load(sim, B["leaves"][I["first_leaf"]:I["first_leaf"] + I["nleaves"]], hmat.store)
    sim.run(B)
    for hmat, I, P in zip(hms, B["instances"], single):
        leaves = B["leaves"][I["first_leaf"]:I["first_leaf"] + I["nleaves"]]
        f = _factor(hmat, sim, leaves)
        one = PlanSim(P["sizes"])
        _load(one, P["leaves"], hmat.store)
        one.run(P)
        g = _factor(hmat, one, P["leaves"])
        A = hmat.exact_dense()
        X = np.random.default_rng(3).standard_normal((hmat.n, 3))
        assert np.linalg.norm(f.apply_lu(X) - g.apply_lu(X)) / np.linalg.norm(A @ X) < 1e-12
        assert np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X) <= 10 * eps


def test_build_then_lu_plans_on_the_host(lib):
    """hm_build's assembly plan (dense leaves evaluated, admissible leaves approximated and
    rounded to eps) gives an H-matrix within eps of the kernel matrix; the H-LU plan run on
    that H-matrix, as hm_lu copies it, gives factors within 10 eps: the device pipeline's data
    flow from points to factors, on the host."""
    from tests.plan_sim import IS_ARANK, SP_A, SP_P
    pts = W.cube_surface(1500, 7)
    eps = 1e-6
    hmat = HMatrix(pts, 64, 2.0, eps, 64)
    S = hm.hm_structure_build(pts, 64, 2.0)
    P = S.plan(6, eps, 64)
    assert len(P["eval"]) and len(P["aca"])
    sim = PlanSim(P["sizes"])
    sim.d[SP_A] = np.zeros(int(P["sizes"]["nvalues"]))
    sim.i[IS_ARANK] = np.zeros(int(P["sizes"]["nranks"]), np.int64)
    sim.d[SP_P] = np.ascontiguousarray(hmat.points[hmat.ct.perm]).ravel()
    sim.h = hmat.h
    sim.run(P)
    A = hmat.exact_dense()
    AH = np.zeros_like(A)
    for lf in P["leaves"]:
        r0, c0 = hmat.ct.clusters[int(lf["row"])].lo, hmat.ct.clusters[int(lf["col"])].lo
        m, n = int(lf["m"]), int(lf["n"])
        if lf["lr"]:
            k = int(sim.i[IS_ARANK][int(lf["rank_idx"])])
            assert 0 < k <= int(lf["cap"])
            U = np.array(sim.mat(ref(SP_A, lf["off"]), 1, m, m, k))
            V = np.array(sim.mat(ref(SP_A, lf["voff"]), 1, n, n, k))
            AH[r0:r0 + m, c0:c0 + n] = U @ V.T
        else:
            AH[r0:r0 + m, c0:c0 + n] = np.array(sim.mat(ref(SP_A, lf["off"]), 1, m, m, n))
    assert np.linalg.norm(A - AH) / np.linalg.norm(A) <= eps
    # the rank of every admissible leaf is the oracle's (its dense SVD truncated at eps)
    for lf in P["leaves"]:
        if lf["lr"]:
            assert int(sim.i[IS_ARANK][int(lf["rank_idx"])]) == hmat.store[(int(lf["row"]), int(lf["col"]))].U.shape[1]
    Q = S.plan(0, eps, 64)
    fac = PlanSim(Q["sizes"])
    fac.d[SP_F] = sim.d[SP_A].copy()
    fac.i[IS_RANK] = sim.i[IS_ARANK].copy()
    fac.run(Q)
    f = _factor(hmat, fac, Q["leaves"])
    X = np.random.default_rng(3).standard_normal((hmat.n, 3))
    assert np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X) <= 10 * eps


@pytest.mark.parametrize("n", [2, 50, 64, 65])
def test_degenerate_sizes_on_the_host(lib, n):
    """One leaf (n <= 64: one LU micro-op, one-leaf solves) and the first split (n = 65): the H-LU
    and solve plans reproduce A and solve with it to rounding."""
    pts = W.fibonacci_sphere(n, 3)
    hmat = HMatrix(pts, 64, 2.0, 1e-6, 64)
    S = hm.hm_structure_build(pts, 64, 2.0)
    P = S.plan(0, 1e-6, 64)
    sim = PlanSim(P["sizes"])
    _load(sim, P["leaves"], hmat.store)
    sim.run(P)
    f = _factor(hmat, sim, P["leaves"])
    A = hmat.exact_dense()
    X = np.random.default_rng(1).standard_normal((n, 2))
    assert np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X) < 1e-14
    Q = S.plan(1, 0.0, 64, 2)
    sol = PlanSim(Q["sizes"], nrhs_space=2 * n)
    sol.d[SP_F], sol.i[IS_RANK], sol.i[IS_PIV] = sim.d[SP_F], sim.i[IS_RANK], sim.i[IS_PIV]
    sol.mat(ref(SP_X, 0), 1, n, n, 2)[:] = X
    sol.i[IS_S][0] = 2
    sol.run(Q)
    xs = np.array(sol.mat(ref(SP_X, 0), 1, n, n, 2))
    assert np.linalg.norm(A @ xs - X) / np.linalg.norm(X) < 1e-13


def _conflicts(fa, fb):
    """Element offsets that one launch group changes and the other accesses, per space."""
    (acc_a, wr_a), (acc_b, wr_b) = fa, fb
    bad = {}
    for wr, acc in ((wr_a, acc_b), (wr_b, acc_a)):
        for key, offs in wr.items():
            hit = np.intersect1d(offs, acc.get(key, np.empty(0, np.int64)))
            if hit.size:
                bad[key] = hit
    return bad


def _merge(fps):
    acc, wr = {}, {}
    for a, w in fps:
        for src, dst in ((a, acc), (w, wr)):
            for k, v in src.items():
                dst[k] = np.union1d(dst.get(k, np.empty(0, np.int64)), v)
    return acc, wr


@pytest.mark.parametrize("which", [7, 9])
def test_overlap_plan_on_the_host(lib, which):
    """The H-LU plan with wave overlap (rounded additions deferred to side launches): the side
    launches of a wave are its last launches and are stack / Gram / core / rebuild launches;
    executed at the latest time the streams allow (after the next wave) they give the same
    factors as in plan order, and the same as the plan without overlap; and no side launch of
    wave w changes memory that a launch of wave w + 1 accesses, or the other way round (the
    two run concurrently on the device). In these task graphs no rounded-addition target of
    wave w is touched by wave w + 1, so every rounded addition is deferred. which = 7: the H-LU
    of Alg 2, 9: the accumulator H-LU (held pieces in the arena)."""
    geom, n, eps = "cube", 700, 1e-6
    pts = W.points_for(geom, n, 21)
    hmat = HMatrix(pts, 64, 2.0, eps, 64)
    S = hm.hm_structure_build(pts, 64, 2.0)
    P0 = S.plan(0 if which == 7 else 8, eps, 64)
    P = S.plan(which, eps, 64)
    L = P["launches"]
    side = L[L["side"] == 1]
    assert side.size > 0 and P["sizes"]["ntrunc"] == P0["sizes"]["ntrunc"]
    assert (P["sizes"]["arena_doubles"] > 0) == (which == 9)
    assert np.all(np.diff(L["wave"]) >= 0)
    assert set(np.unique(side["kind"]).tolist()) <= {4, 5, 2}   # stack, core, gemm
    for w in np.unique(side["wave"]):
        idx = np.flatnonzero(L["wave"] == w)
        flags = L["side"][idx]
        assert np.all(np.diff(flags) >= 0), f"wave {w}: a side launch before one of the wave's others"
    spaces = set()
    for t in ("gemm", "trunc"):
        for f in P[t].dtype.names:
            if P[t].dtype[f] == np.uint64:
                spaces |= set((P[t][f][P[t][f] != 0] >> 60).astype(int).tolist())
    assert 6 in spaces, "no reference into the second scratch space"   # SP_S2 + 1

    runs = []
    for order in (None, PlanSim.latest_order(L)):
        sim = PlanSim(P["sizes"])
        _load(sim, P["leaves"], hmat.store)
        sim.run(P, order)
        runs.append(sim)
    base = PlanSim(P0["sizes"])
    _load(base, P0["leaves"], hmat.store)
    base.run(P0)
    assert np.array_equal(runs[0].d[SP_F], runs[1].d[SP_F])
    assert np.array_equal(runs[0].i[IS_RANK], runs[1].i[IS_RANK])
    A = hmat.exact_dense()
    X = np.random.default_rng(5).standard_normal((n, 3))
    f = _factor(hmat, runs[1], P["leaves"])
    g = _factor(hmat, base, P0["leaves"])
    assert np.linalg.norm(f.apply_lu(X) - g.apply_lu(X)) / np.linalg.norm(A @ X) < 1e-13
    assert np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X) <= 10 * eps

    # footprints: run in plan order, recording each side group and the next wave's launches
    sim = PlanSim(P["sizes"])
    _load(sim, P["leaves"], hmat.store)
    waves_with_side = set(np.unique(side["wave"]).tolist())
    groups = {}
    for ln in L:
        w, sd = int(ln["wave"]), int(ln["side"])
        if (sd and w in waves_with_side) or (not sd and (w - 1 in waves_with_side or w - 2 in waves_with_side)):
            groups.setdefault((w, sd), []).append(sim.footprint(P, ln))
        else:
            sim.run_launch(P, ln)
    checked = later = 0
    for w in waves_with_side:
        if (w + 1, 0) in groups:
            bad = _conflicts(_merge(groups[(w, 1)]), _merge(groups[(w + 1, 0)]))
            assert not bad, f"wave {w}: side launches and wave {w + 1} share {list(bad)}"
            checked += 1
        if (w + 2, 0) in groups:
            later += bool(_conflicts(_merge(groups[(w, 1)]), _merge(groups[(w + 2, 0)])))
    # the check sees real dependences: wave w + 2 reuses the scratch of wave w's side launches
    # and updates some of their targets again, which is why it waits for them
    assert checked > 0 and later > 0


class _CountingAccu:
    """The oracle's accumulator H-LU (piece lists), recording how many pieces every low-rank
    leaf receives in its one rounded addition."""

    @staticmethod
    def run(hmat):
        from oracle.accu import AccuHLUFactor

        class Rec(AccuHLUFactor):
            def apply_to_leaf(self, leaf, alpha, pieces, base_row, base_col):
                lr0, lr1 = leaf.row.lo - base_row, leaf.row.hi - base_row
                lc0, lc1 = leaf.col.lo - base_col, leaf.col.hi - base_col
                k = sum(1 for (r0, c0, Wp, Zp) in pieces
                        if max(r0, lr0) < min(r0 + Wp.shape[0], lr1) and max(c0, lc0) < min(c0 + Zp.shape[0], lc1))
                if k and not isinstance(self.M[leaf.key], Dense):
                    self.counts[(leaf.row.lo, leaf.col.lo)] = self.counts.get((leaf.row.lo, leaf.col.lo), 0) + k
                return super().apply_to_leaf(leaf, alpha, pieces, base_row, base_col)

        R = Rec(hmat)
        R.counts = {}
        return R.factor()


@pytest.mark.parametrize("geom,n,eps", [("sphere", 1024, 1e-6), ("cube", 1500, 1e-4)])
def test_accumulator_plan_on_the_host(lib, geom, n, eps):
    """The accumulator H-LU plan (Alg 4-8, piece lists): every low-rank leaf receives in its
    rounded additions exactly the pieces that the oracle's accumulator H-LU hands to it in one
    apply_upd (counted per leaf, through the trees of rounded additions that large stacks
    take), fewer rounded additions than the H-LU of Alg 2, and factors within 10 eps of the
    exact kernel and within eps of the oracle's accumulator factors."""
    pts = W.points_for(geom, n, 21)
    hmat = HMatrix(pts, 64, 2.0, eps, 64)
    S = hm.hm_structure_build(pts, 64, 2.0)
    P0 = S.plan(0, eps, 64)
    P = S.plan(8, eps, 64)
    assert P["sizes"]["arena_doubles"] > 0
    assert P["sizes"]["ntrunc"] < P0["sizes"]["ntrunc"]
    R = _CountingAccu.run(hmat)
    cl = S.export()["clusters"]
    key = {int(lf["off"]): (int(cl[lf["row"], 0]), int(cl[lf["col"], 0])) for lf in P["leaves"] if lf["lr"]}
    # the pieces of every rounded addition, followed through the temporary sums of the trees of
    # rounded additions (a stack without self writes a sum that a later stack takes as an entry;
    # scratch addresses repeat from wave to wave, so a sum is identified by wave and address)
    L = P["launches"]
    ops = [(int(ln["wave"]), op) for ln in L[L["kind"] == 4]
           for op in P["trunc"][ln["begin"]:ln["begin"] + ln["count"]]]
    ents = lambda op: P["entries"][int(op["first_entry"]):int(op["first_entry"]) + int(op["n_entries"])]
    sums = {(w, int(op["U"])) for w, op in ops if int(op["flags"]) & 1}
    assert sums, "no tree of rounded additions in this plan"
    consumer = {(w, int(e["W"])): q for q, (w, op) in enumerate(ops) for e in ents(op) if (w, int(e["W"])) in sums}
    counts = {}
    for w, op in ops:
        out = op
        while int(out["flags"]) & 1:
            out = ops[consumer[(w, int(out["U"]))]][1]
        k = key[int(out["U"]) & ((1 << 60) - 1)]
        counts[k] = counts.get(k, 0) + sum(1 for e in ents(op) if (w, int(e["W"])) not in sums)
    assert counts == R.counts
    sim = PlanSim(P["sizes"])
    _load(sim, P["leaves"], hmat.store)
    sim.run(P)
    assert sim.singular == 0
    f = _factor(hmat, sim, P["leaves"])
    A = hmat.exact_dense()
    X = np.random.default_rng(3).standard_normal((n, 4))
    AX = A @ X
    assert np.linalg.norm(AX - f.apply_lu(X)) / np.linalg.norm(AX) <= 10 * eps
    assert np.linalg.norm(f.apply_lu(X) - R.apply_lu(X)) / np.linalg.norm(AX) <= eps
