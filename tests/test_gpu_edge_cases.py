"""Edge cases and failure paths of the CUDA path (GPU; every call goes through the C ABI).

* partial pivoting inside the leaf LU (row interchanges, and P^T applied by the solves): the
  kernel matrix 1/(r + h) keeps its largest entry of every column on the diagonal, so the
  rows of every leaf block are permuted inside their leaf cluster, as for the oracle's own
  pivoting pin; compared with the oracle on the same permuted matrix;
* the rank cap (rounded additions that keep at most `cap` singular values) and stacks of
  numerical rank above 128 (the FP64 two-sided Jacobi branch of the truncation core);
* the accuracy floor: eps below HM_EPS_MIN is rejected instead of silently missed;
* numerically singular leaves (duplicate points) report HM_ESINGULAR with the factor returned;
* an allocator that fails at any one of its calls gives HM_ENOMEM, leaks nothing, and the
  next calls succeed;
* the FP64 reciprocal helpers of the serial sections against IEEE division / square root;
* batching across instances, the GEMM split autotuner, and the wave overlap of deferred
  rounded additions against the sequential schedule.
"""
import numpy as np
import pytest

import hm_workloads as W
from oracle.geometry import kernel_block, mean_nn_spacing
from oracle.hlu import HLUFactor
from oracle.hmatrix import HMatrix, LowRank, truncate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_07531_gb300 as hm
    hm.build_library()
    return hm


@pytest.fixture(scope="module")
def ctx(hm):
    return hm.HMContext(0)


def dev(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda() if a.ndim == 1 else \
        torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def host(t):
    return t.detach().cpu().numpy()


def fro_ratio(E, R):
    return float(np.linalg.norm(E) / np.linalg.norm(R))


# ------------------------------------------------------------------ partial pivoting
def _leaf_row_permutation(lay, seed):
    """pi over cluster positions: a random permutation inside every leaf cluster."""
    leaves, lo = lay["leaves"], lay["cluster_lo"]
    n = len(lay["perm"])
    pi = np.arange(n)
    rng = np.random.default_rng(seed)
    seen = set()
    for row, col, m, *_ in leaves:
        if row == col and row not in seen:          # diagonal leaves cover the leaf clusters
            seen.add(row)
            a = lo[row]
            pi[a:a + m] = a + rng.permutation(m)
    return pi


def _permute_device_values(A, lay, pi):
    """Rows of every leaf block (dense D, or U of U V^T) permuted by pi, on the device."""
    vals = A.get_values()
    lo = lay["cluster_lo"]
    for row, col, m, n, lr, cap, off, voff, ridx, poff in lay["leaves"]:
        loc = torch.from_numpy(pi[lo[row]:lo[row] + m] - lo[row]).cuda()
        ncol = cap if lr else n
        blk = vals[off:off + m * ncol].view(ncol, m)     # column-major m x ncol
        vals[off:off + m * ncol] = blk[:, loc].reshape(-1)
    A.set_values(vals)


def _permute_oracle_values(o, pi):
    for b in o.bt.leaves():
        st = o.store[b.key]
        loc = pi[b.row.lo:b.row.hi] - b.row.lo
        if isinstance(st, LowRank):
            st.U = st.U[loc]
        else:
            st.D = st.D[loc]


@pytest.mark.parametrize("geom,n,eta,eps", [("cube", 700, 0.0, 1e-8), ("cube", 1500, 2.0, 1e-6),
                                            ("sphere", 2048, 2.0, 1e-4)])
def test_lu_with_row_interchanges(ctx, hm, geom, n, eta, eps):
    """P L U of the leaf-row-permuted matrix: interchanges happen (counted by the kernel), the
    factorization error of the permuted matrix is within 10 eps (all dense: 1e-13) and within
    10x the oracle's on the same permuted matrix, and a refined solve matches a dense solve."""
    p = W.points_for(geom, n, 9)
    A = hm.hm_build(ctx, p, 64, eta, eps, 64)
    lay = A.layout()
    pi = _leaf_row_permutation(lay, 1)
    assert np.any(pi != np.arange(n))
    _permute_device_values(A, lay, pi)
    F = hm.hm_lu(ctx, A)
    st = F.stats()
    assert st["row_interchanges"] > 0
    assert st["singular_pivots"] == 0
    perm = lay["perm"]
    # (Pi A x) in original order: row perm[i] of the result is row perm[pi[i]] of A x
    X = np.random.default_rng(5).standard_normal((n, 6))
    Xd = dev(X)
    Ax = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, Xd))
    PAx = np.empty_like(Ax)
    PAx[perm] = Ax[perm[pi]]
    LUx = host(hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F))
    err = fro_ratio(LUx - PAx, PAx)
    if eta == 0.0:
        assert err < 1e-13
    else:
        assert err <= 10 * eps
        o = HMatrix(p, 64, eta, eps, 64)
        _permute_oracle_values(o, pi)
        of = HLUFactor(o).factor()
        Aex = o.exact_dense()[pi]                     # cluster order, rows permuted
        Xp = X[perm]
        oerr = fro_ratio(Aex @ Xp - of.apply_lu(Xp), Aex @ Xp)
        assert oerr <= 10 * eps
        assert err <= 10 * max(oerr, 1e-15)
    # solve of the permuted system against a dense solve (original order)
    h = A.stats()["h"]
    K = kernel_block(p, p, h)
    Kp = np.empty_like(K)
    Kp[perm] = K[perm[pi]]
    b = np.random.default_rng(6).standard_normal(n)
    x, _ = hm.hm_solve(ctx, F, dev(b))
    xe = np.linalg.solve(Kp, b)
    assert np.linalg.norm(host(x) - xe) / np.linalg.norm(xe) < (1e-11 if eta == 0.0 else 1e3 * eps)


# ------------------------------------------------------------------ rank cap, wide stacks
def test_rank_cap_hits_match_oracle(ctx, hm):
    """sphere 2048 at eps 1e-8 with rank cap 8: the cap decides most truncations; the GPU's
    error is that of the oracle with the same cap, within 10x."""
    p = W.fibonacci_sphere(2048, 11)
    A = hm.hm_build(ctx, p, 64, 2.0, 1e-8, 8)
    F = hm.hm_lu(ctx, A)
    st = F.stats()
    assert st["rank_cap_hits"] > 0
    assert st["max_rank"] <= 8
    X = np.random.default_rng(5).standard_normal((2048, 8))
    Xd = dev(X)
    Ax = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, Xd))
    err = fro_ratio(host(hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F)) - Ax, Ax)
    o = HLUFactor(HMatrix(p, 64, 2.0, 1e-8, 8)).factor()
    Ao = o.hm.exact_dense()
    oerr = fro_ratio(Ao @ X - o.apply_lu(X), Ao @ X)
    assert oerr > 1e-6                      # the cap, not eps, sets the error
    assert err <= 10 * oerr


def test_truncate_wide_stack_two_sided_jacobi(ctx, hm):
    """A stack of 200 columns with numerical rank 200 (> 128: FP64 two-sided Jacobi branch),
    cap 64: the result is the best rank-64 approximation up to the Gram floor."""
    m = n = 600
    r = 200
    rng = np.random.default_rng(3)
    s = np.logspace(0, -5, r)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, r)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, r)))
    Qm, _ = np.linalg.qr(rng.standard_normal((r, r)))
    Mx = Qm @ np.diag(np.logspace(0, 1, r))
    Wm = (Q1 * s) @ Mx
    Zm = Q2 @ np.linalg.inv(Mx).T
    exact = Q1 @ np.diag(s) @ Q2.T
    for eps in (1e-4, 1e-6):
        U, V = hm.hm_truncate(ctx, dev(Wm), dev(Zm), eps, 64)
        assert U.shape[1] == 64
        err = np.linalg.norm(host(U) @ host(V).T - exact, 2)
        assert err <= s[64] + 1e-7 * s[0]
        Uo, Vo = truncate(Wm, Zm, eps, 64)
        assert Uo.shape[1] == 64
        assert np.linalg.norm(Uo @ Vo.T - exact, 2) <= s[64] * (1 + 1e-6)


# ------------------------------------------------------------------ accuracy floor
def test_eps_below_floor_is_rejected(ctx, hm):
    p = W.fibonacci_sphere(300, 1)
    with pytest.raises(hm.HMError, match="HM_EINVAL"):
        hm.hm_build(ctx, p, 64, 2.0, 1e-9, 64)
    A = hm.hm_build(ctx, p, 64, 2.0, 1e-8, 64)
    with pytest.raises(hm.HMError, match="HM_EINVAL"):
        hm.hm_lu(ctx, A, eps=1e-10)
    with pytest.raises(hm.HMError, match="HM_EINVAL"):
        hm.hm_truncate(ctx, dev(np.ones((10, 2))), dev(np.ones((8, 2))), 5e-9, 64)
    with pytest.raises(hm.HMError, match="HM_EINVAL"):
        hm.hm_truncate_noalloc(dev(np.ones((10, 2))), dev(np.ones((8, 2))), 5e-9, 64)


# ------------------------------------------------------------------ singular leaves
def test_duplicate_points_report_singular(ctx, hm):
    """Two copies of one point give two equal rows: the leaf LU meets a numerically zero pivot,
    hm_lu returns HM_ESINGULAR, and the factor is still returned with the count."""
    base = W.fibonacci_sphere(63, 4)
    p = np.vstack([base, base[17:18]])              # 64 points: one leaf, one dense LU
    A = hm.hm_build(ctx, p, 64, 0.0, 1e-8, 64)
    with pytest.raises(hm.HMError, match="HM_ESINGULAR"):
        hm.hm_lu(ctx, A)
    F = hm.hm_lu(ctx, A, allow_singular=True)
    assert F is not None and F.stats()["singular_pivots"] >= 1
    # a regular matrix of the same size reports none
    A2 = hm.hm_build(ctx, base, 64, 0.0, 1e-8, 64)
    assert hm.hm_lu(ctx, A2).stats()["singular_pivots"] == 0


def test_duplicate_points_in_first_leaf_of_h_matrix(ctx, hm):
    """The same in an H-matrix: the copy lands in the first leaf cluster (checked on the
    cluster order), whose LU runs first on the assembled values."""
    base = W.cube_surface(1000, 5)
    s0 = hm.hm_structure_build(base, 64, 2.0).export()
    i0 = int(s0["perm"][0])
    p = np.vstack([base, base[i0:i0 + 1]])
    A = hm.hm_build(ctx, p, 64, 2.0, 1e-6, 64)
    lay = A.layout()
    first = lay["leaves"][0]
    assert first[0] == first[1]                      # the first leaf is a diagonal leaf
    pos = {int(v): k for k, v in enumerate(lay["perm"])}
    assert pos[i0] < first[2] and pos[1000] < first[2]
    F = hm.hm_lu(ctx, A, allow_singular=True)
    assert F.stats()["singular_pivots"] >= 1


# ------------------------------------------------------------------ allocation failures
def test_allocation_failure_at_every_call(hm):
    """An allocator that returns NULL at its k-th call, for every k of a build -> LU -> solve
    (with refinement) -> matvec sequence: the failing call raises HM_ENOMEM, nothing the
    library allocated stays allocated once the handles are freed, and the same sequence then
    runs with a working allocator to the same result."""
    p = W.cube_surface(400, 2)
    b = np.random.default_rng(1).standard_normal(400)
    state = {"calls": 0, "fail_at": -1}

    def admit(nbytes):
        state["calls"] += 1
        return state["calls"] != state["fail_at"]

    c = hm.HMContext(0, admit=admit)

    def sequence():
        A = F = None
        try:
            A = hm.hm_build(c, p, 64, 2.0, 1e-6, 64)
            F = hm.hm_lu(c, A)
            x, _ = hm.hm_solve(c, F, dev(b), A=A, refine_tol=1e-10, max_iter=10, residual_op=hm.HM_OP_EXACT)
            y = hm.hm_matvec(c, A, hm.HM_OP_A, x)
            return host(x), host(y)
        finally:
            if F is not None:
                F.free()
            if A is not None:
                A.free()

    torch.cuda.synchronize()
    base_mem = torch.cuda.memory_allocated()
    x_ref, y_ref = sequence()
    ncalls = state["calls"]
    assert ncalls > 10
    assert torch.cuda.memory_allocated() == base_mem
    failures = 0
    for k in range(1, ncalls + 1):
        state.update(calls=0, fail_at=k)
        try:
            sequence()
        except hm.HMError as ex:
            assert ex.code == -2, str(ex)
            failures += 1
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base_mem, f"leak after a failure at call {k}"
    assert failures == ncalls
    state.update(calls=0, fail_at=-1)
    x2, y2 = sequence()
    assert np.linalg.norm(x2 - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert np.linalg.norm(y2 - y_ref) <= 1e-9 * np.linalg.norm(y_ref)


# ------------------------------------------------------------------ reciprocal helpers
def _ulps(got, ref):
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_reciprocal_helpers_against_ieee(hm):
    rng = np.random.default_rng(12)
    mant = rng.uniform(1.0, 2.0, 20000)
    wide = mant * 2.0 ** rng.integers(-1000, 1000, mant.size)          # normal range
    mid = mant * 2.0 ** rng.integers(-95, 95, mant.size)                # inside [1e-30, 1e30]
    edge = np.concatenate([np.nextafter(1e-30, 0) * np.array([1.0, 1 + 1e-15]), [1e-30, 1e30],
                           np.nextafter(1e30, np.inf) * np.array([1.0, 1 - 1e-15]), [1.0, 0.5, 2.0, 3.0]])
    sgn = np.where(rng.random(mant.size) < 0.5, -1.0, 1.0)
    cases = {
        0: np.concatenate([wide * sgn, edge, -edge]),                   # nr_rcp
        1: np.concatenate([wide, edge]),                                 # nr_rsqrt
        2: np.concatenate([mid, edge[2:4]]),                             # fast_rcp
        3: np.concatenate([wide * sgn, mid * sgn, edge, -edge]),         # pivot reciprocal
    }
    for which, x in cases.items():
        y = host(hm.hm_selftest_reciprocals(dev(x), which))
        ref = 1.0 / np.sqrt(x) if which == 1 else 1.0 / x
        u = _ulps(y, ref)
        assert u.max() <= 2.0, (which, float(u.max()), float(x[np.argmax(u)]))
    with pytest.raises(hm.HMError, match="HM_EINVAL"):
        hm.hm_selftest_reciprocals(dev(np.ones(3)), 4)


# ------------------------------------------------------------------ batching across instances
def test_lu_batch_matches_solo_factors(ctx, hm):
    """hm_lu_batch over three instances of different n: each factor within 10 eps of its exact
    kernel matrix, each solve equal to its own hm_lu's solve within the tolerance of the
    factorization; factors freed in an order different from creation (shared arena)."""
    eps = 1e-6
    pts = [W.ellipsoid(n, 100 + n) for n in (1100, 2048, 1500)]
    mats = [hm.hm_build(ctx, p, 64, 2.0, eps, 64) for p in pts]
    Fs = hm.hm_lu_batch(ctx, mats)
    assert len(Fs) == 3 and all(F is not None for F in Fs)
    xs = []
    for A, F, p in zip(mats, Fs, pts):
        n = p.shape[0]
        X = np.random.default_rng(5).standard_normal((n, 4))
        Xd = dev(X)
        Ax = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, Xd))
        err = fro_ratio(host(hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F)) - Ax, Ax)
        assert err <= 10 * eps
        b = np.random.default_rng(n).standard_normal(n)
        xb, _ = hm.hm_solve(ctx, F, dev(b))
        Fs1 = hm.hm_lu(ctx, A)
        x1, _ = hm.hm_solve(ctx, Fs1, dev(b))
        Fs1.free()
        xe = np.linalg.solve(kernel_block(p, p, A.stats()["h"]), b)
        e_b = np.linalg.norm(host(xb) - xe) / np.linalg.norm(xe)
        e_1 = np.linalg.norm(host(x1) - xe) / np.linalg.norm(xe)
        assert e_b <= 10 * max(e_1, 1e-12)
        assert np.linalg.norm(host(xb) - host(x1)) / np.linalg.norm(host(x1)) <= 10 * max(e_1, 1e-12)
        xs.append(host(xb))
    for i in (1, 0, 2):                               # free out of creation order
        Fs[i].free()
    for A in mats:
        A.free()


# ------------------------------------------------------------------ GEMM split autotuner
def test_autotune_gemm_split(ctx, hm):
    """The autotuner times hm_lu at every candidate split target, keeps the fastest set; the
    factorization stays within 10 eps at every setting."""
    p = W.fibonacci_sphere(4096, 3)
    A = hm.hm_build(ctx, p, 64, 2.0, 1e-6, 64)
    before = hm.hm_get_gemm_work()
    try:
        best, times = hm.hm_autotune_gemm(ctx, A, candidates=(4096.0, 16384.0, 65536.0))
        assert best in times and all(t > 0 for t in times.values())
        assert times[best] == min(times.values())
        assert hm.hm_get_gemm_work() == best
        for w in (4096.0, 65536.0):
            hm.hm_set_gemm_work(w)
            F = hm.hm_lu(ctx, A)
            X = np.random.default_rng(5).standard_normal((4096, 4))
            Xd = dev(X)
            Ax = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, Xd))
            assert fro_ratio(host(hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F)) - Ax, Ax) <= 1e-5
            F.free()
    finally:
        hm.hm_set_gemm_work(before)


# ------------------------------------------------------------------ wave overlap
def test_wave_overlap_matches_sequential(ctx, hm):
    """Rounded additions deferred to the side stream (hm_set_overlap(1)) give the factors of
    the sequential schedule (hm_set_overlap(0)) up to the order of atomic accumulations, and
    a profiled factorization (sequential by construction) agrees too: all within 10 eps of the
    exact kernel and within eps of each other."""
    n, eps = 8192, 1e-6
    p = W.cube_surface(n, 31)
    A = hm.hm_build(ctx, p, 64, 2.0, eps, 64)
    X = np.random.default_rng(7).standard_normal((n, 4))
    Xd = dev(X)
    Ax = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, Xd))
    before = hm.hm_get_overlap()
    out = {}
    try:
        for on, prof in ((1, False), (0, False), (1, True)):
            hm.hm_set_overlap(on)
            assert hm.hm_get_overlap() == on
            ctx.set_profiling(prof)
            F = hm.hm_lu(ctx, A)
            ctx.set_profiling(False)
            out[(on, prof)] = host(hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F))
            assert fro_ratio(out[(on, prof)] - Ax, Ax) <= 10 * eps
            F.free()
        with pytest.raises(hm.HMError, match="HM_EINVAL"):
            hm.hm_set_overlap(2)
    finally:
        ctx.set_profiling(False)
        hm.hm_set_overlap(before)
    ref = out[(0, False)]   # rank decisions near eps may differ with the accumulation order
    assert fro_ratio(out[(1, False)] - ref, Ax) <= eps
    assert fro_ratio(out[(1, True)] - ref, Ax) <= eps


# ------------------------------------------------------------------ H-LU prepared during the build
def test_prepare_lu_during_build(ctx, hm):
    """hm_build with prepare_lu plans the H-LU on a host thread during the assembly: hm_lu then
    factors with that plan (no planning left: its plan time is the thread's), the factor equals
    one planned by hm_lu itself within rounding of the atomic accumulations, a different eps
    re-plans, and freeing the matrix without factoring it waits for the thread."""
    n, eps = 4096, 1e-6
    p = W.fibonacci_sphere(n, 9)
    X = np.random.default_rng(8).standard_normal((n, 3))
    A0 = hm.hm_build(ctx, p, 64, 2.0, eps, 64)
    A1 = hm.hm_build(ctx, p, 64, 2.0, eps, 64, prepare_lu=True)
    s1 = A1.stats()   # waits for the preparation
    assert s1["dag_levels"] > 0 and s1["plan_launches"] > 0
    F0, F1 = hm.hm_lu(ctx, A0), hm.hm_lu(ctx, A1)
    assert F1.stats()["plan_launches"] == F0.stats()["plan_launches"]
    Xd = dev(X)
    Ax = host(hm.hm_matvec(ctx, A0, hm.HM_OP_EXACT, Xd))
    y0 = host(hm.hm_matvec(ctx, A0, hm.HM_OP_LU, Xd, F=F0))
    y1 = host(hm.hm_matvec(ctx, A1, hm.HM_OP_LU, Xd, F=F1))
    assert fro_ratio(y1 - Ax, Ax) <= 10 * eps
    assert fro_ratio(y1 - y0, Ax) <= eps
    F2 = hm.hm_lu(ctx, A1, eps=1e-4)   # another eps: planned again
    assert fro_ratio(host(hm.hm_matvec(ctx, A1, hm.HM_OP_LU, Xd, F=F2)) - Ax, Ax) <= 1e-3
    for F in (F0, F1, F2):
        F.free()
    A0.free()
    A1.free()
    A3 = hm.hm_build(ctx, p, 64, 2.0, eps, 64, prepare_lu=True)
    A3.free()   # joins the preparation thread
