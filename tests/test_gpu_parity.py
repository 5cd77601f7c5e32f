"""Parity of the CUDA path against the FP64 oracle (GPU; calls go through the C ABI).

Floating-point results are compared by what is unique: reconstruction errors against exact
kernel matrices, ranks from known singular values, the relative factorization error
||A - P L U|| / ||A|| <= 10 eps (the stated tolerance), and solve accuracy; never factor by
factor (H-LU factors are not unique up to the truncations' rotations).
"""
import math

import numpy as np
import pytest

import hm_workloads as W
from oracle.geometry import kernel_block, kernel_matvec_rows, mean_nn_spacing
from oracle.hlu import HLUFactor
from oracle.hmatrix import HMatrix, truncate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_07531_gb300 as hm
    hm.build_library()
    return hm.HMContext(0)


@pytest.fixture(scope="module")
def hm():
    import paper_1911_07531_gb300 as hm
    return hm


def dev(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda() if a.ndim == 1 else \
        torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def host(t):
    return t.detach().cpu().numpy()


def fro_ratio(E, R):
    return float(np.linalg.norm(E) / np.linalg.norm(R))


# ------------------------------------------------------------------ rounded truncation (K8)
@pytest.mark.parametrize("m,n,K", [(90, 70, 7), (700, 513, 40), (64, 64, 128), (3000, 100, 200), (5, 9, 3)])
def test_truncate_matches_known_singular_values(ctx, hm, m, n, K):
    """W Z^T with known singular values, split into non-orthogonal factors (mixing of condition
    10) padded with redundant columns. Gram-based truncation keeps sigma_i > eps sigma_1 like the
    oracle; its accuracy floor is about sqrt(K u) |W| |Z|, so the bound is tail + 1e-7 sigma_1."""
    rng = np.random.default_rng(m + n + K)
    r = min(K, m, n)
    s = np.logspace(0, -12.37, r)   # exponents off the thresholds eps = 1e-4, 1e-6
    Q1, _ = np.linalg.qr(rng.standard_normal((m, r)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, r)))
    Qm, _ = np.linalg.qr(rng.standard_normal((r, r)))
    Mx = Qm @ np.diag(np.logspace(0, 1, r))
    Wm = (Q1 * s) @ Mx
    Zm = Q2 @ np.linalg.inv(Mx).T
    if K > r:
        Wm = np.hstack([Wm, np.zeros((m, K - r))])
        Zm = np.hstack([Zm, rng.standard_normal((n, K - r))])
    exact = Q1 @ np.diag(s) @ Q2.T
    for eps in (1e-4, 1e-6):
        U, V = hm.hm_truncate(ctx, dev(Wm), dev(Zm), eps, 64)
        k_ref = min(64, int(np.count_nonzero(s > eps * s[0])))
        Uo, Vo = truncate(Wm, Zm, eps, 64)
        assert Uo.shape[1] == k_ref
        assert U.shape[1] == k_ref
        Uh, Vh = host(U), host(V)
        tail = s[k_ref] if k_ref < r else 0.0
        err = np.linalg.norm(Uh @ Vh.T - exact, 2)
        assert err <= tail + 1e-7 * s[0]
        assert np.linalg.norm(Uo @ Vo.T - exact, 2) <= tail * (1 + 1e-6) + 1e-13


def test_truncate_zero_and_edge(ctx, hm):
    U, V = hm.hm_truncate(ctx, dev(np.zeros((10, 4))), dev(np.ones((7, 4))), 1e-6, 64)
    assert U.shape[1] == 0
    U, V = hm.hm_truncate(ctx, dev(np.ones((1, 1))), dev(np.full((1, 1), 2.0)), 1e-6, 64)
    assert U.shape[1] == 1 and abs(host(U)[0, 0] * host(V)[0, 0] - 2.0) < 1e-14
    with pytest.raises(hm.HMError):
        hm.hm_truncate(ctx, dev(np.ones((4, 300))), dev(np.ones((4, 300))), 1e-6, 64)


# ------------------------------------------------------------------ build + matvec
def test_build_and_matvec_against_exact_kernel(ctx, hm):
    p = W.fibonacci_sphere(2048, 11)
    A = hm.hm_build(ctx, p, 64, 2.0, 1e-8, 64)
    st = A.stats()
    assert st["h"] == pytest.approx(mean_nn_spacing(p), rel=1e-13)
    assert st["nleaves_lowrank"] > 0 and st["aca_unconverged"] == 0
    x = np.random.default_rng(2).standard_normal((2048, 3))
    Ax = kernel_block(p, p, st["h"]) @ x
    y = host(hm.hm_matvec(ctx, A, hm.HM_OP_A, dev(x)))
    assert fro_ratio(y - Ax, Ax) < 1e-7
    ye = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, dev(x)))
    assert fro_ratio(ye - Ax, Ax) < 1e-13
    # alpha / beta semantics
    y0 = np.random.default_rng(3).standard_normal((2048, 3))
    y2 = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, dev(x), dev(y0), alpha=2.0, beta=-0.5))
    assert fro_ratio(y2 - (2 * Ax - 0.5 * y0), Ax) < 1e-13


# ------------------------------------------------------------------ H-LU
def _lu_error(ctx, hm, A, F, n, ncol=8, seed=5):
    X = np.random.default_rng(seed).standard_normal((n, ncol))
    Xd = dev(X)
    Ax = hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, Xd)
    LUx = hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F)
    return fro_ratio(host(Ax) - host(LUx), host(Ax))


def test_lu_all_dense_equals_dense_lu(ctx, hm):
    p = W.fibonacci_sphere(300, 2)
    A = hm.hm_build(ctx, p, 64, 0.0, 1e-8, 64)
    F = hm.hm_lu(ctx, A)
    assert _lu_error(ctx, hm, A, F, 300) < 1e-14
    b = np.random.default_rng(4).standard_normal(300)
    x, _ = hm.hm_solve(ctx, F, dev(b))
    h = A.stats()["h"]
    xe = np.linalg.solve(kernel_block(p, p, h), b)
    assert np.linalg.norm(host(x) - xe) / np.linalg.norm(xe) < 1e-12
    # L and U separately: P L U x == L-op(U-op(x))
    Xd = dev(np.random.default_rng(1).standard_normal((300, 2)))
    u = hm.hm_matvec(ctx, A, hm.HM_OP_U, Xd, F=F)
    lu2 = hm.hm_matvec(ctx, A, hm.HM_OP_L, u, F=F)
    lu = hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F)
    assert fro_ratio(host(lu2) - host(lu), host(lu)) < 1e-14


@pytest.mark.parametrize("geom,n,eps", [("sphere", 2048, 1e-4), ("cube", 3000, 1e-6), ("sphere", 1024, 1e-8)])
def test_lu_within_ten_eps_and_oracle(ctx, hm, geom, n, eps):
    """||A - P L U|| / ||A|| <= 10 eps for eps >= 1e-8. The GPU's rounded truncation forms Gram
    matrices of the stacked factors, so its accuracy floor is about sqrt(K u) ~ 1e-8 relative to
    the stacked factors (3.8e-9 was measured at eps = 1e-10, n = 1024); smaller eps is not
    claimed."""
    p = W.points_for(geom, n, 11)
    A = hm.hm_build(ctx, p, 64, 2.0, eps, 64)
    F = hm.hm_lu(ctx, A)
    st = F.stats()
    assert st["singular_pivots"] == 0
    err = _lu_error(ctx, hm, A, F, n)
    assert err <= 10 * eps
    if n <= 2048:
        o = HLUFactor(HMatrix(p, 64, 2.0, eps, 64)).factor()
        X = np.random.default_rng(5).standard_normal((n, 8))
        Ao = o.hm.exact_dense()
        oerr = fro_ratio(Ao @ X - o.apply_lu(X), Ao @ X)
        assert oerr <= 10 * eps
        assert err <= 10 * max(oerr, 1e-15)
    # refinement against the exact kernel reaches 1e-10 residual; error vs dense solve
    b = np.random.default_rng(6).standard_normal((n, 2))
    x, info = hm.hm_solve(ctx, F, dev(b), A=A, refine_tol=1e-10, max_iter=30, residual_op=hm.HM_OP_EXACT)
    assert info["rel_residual"] <= 1e-10
    xe = np.linalg.solve(kernel_block(p, p, A.stats()["h"]), b)
    assert np.linalg.norm(host(x) - xe) / np.linalg.norm(xe) < 1e-8


def test_solve_many_rhs_and_alias(ctx, hm):
    """70 right-hand sides (three 32-column chunks) equal 70 single solves; in-place solve equals
    the out-of-place one; accuracy within the claimed range (eps = 1e-8), and 1e-10 with
    refinement against the exact kernel."""
    p = W.cube_surface(1500, 3)
    A = hm.hm_build(ctx, p, 64, 2.0, 1e-8, 64)
    F = hm.hm_lu(ctx, A)
    B = np.random.default_rng(7).standard_normal((1500, 70))
    X, _ = hm.hm_solve(ctx, F, dev(B))
    Xh = host(X)
    for j in (0, 31, 32, 69):
        xj, _ = hm.hm_solve(ctx, F, dev(B[:, j].copy()))
        assert np.linalg.norm(host(xj) - Xh[:, j]) <= 1e-13 * np.linalg.norm(Xh[:, j])
    xe = np.linalg.solve(kernel_block(p, p, A.stats()["h"]), B)
    assert fro_ratio(Xh - xe, xe) < 1e-5
    Bd = dev(B)
    hm.hm_solve(ctx, F, Bd, Bd)                                  # in place
    assert fro_ratio(host(Bd) - Xh, Xh) < 1e-14
    Xr, info = hm.hm_solve(ctx, F, dev(B[:, :3].copy()), A=A, refine_tol=1e-12, max_iter=20,
                           residual_op=hm.HM_OP_EXACT)
    assert info["rel_residual"] <= 1e-12
    assert fro_ratio(host(Xr) - xe[:, :3], xe[:, :3]) < 1e-10


def test_invalid_arguments_fail_loudly(ctx, hm):
    with pytest.raises(hm.HMError):
        hm.hm_build(ctx, np.zeros((0, 3)))
    with pytest.raises(hm.HMError):
        hm.hm_build(ctx, W.fibonacci_sphere(100, 1), rank_cap=65)
    A = hm.hm_build(ctx, W.fibonacci_sphere(200, 1))
    with pytest.raises(hm.HMError):
        hm.hm_matvec(ctx, A, hm.HM_OP_LU, dev(np.ones(200)))     # needs a factor


# ------------------------------------------------------------------ full size (sampled)
@pytest.mark.slow
def test_full_size_cube_sampled_rows(ctx, hm):
    """n = 131072 cube surface, eps = 1e-6: rows of (A - P L U) x checked one by one."""
    cfg = W.WORKLOADS["cube131072"]
    p = W.points_for(cfg["geometry"], cfg["n"], cfg["seed"])
    A = hm.hm_build(ctx, p, cfg["leaf"], cfg["eta"], cfg["eps"], cfg["rank_cap"])
    F = hm.hm_lu(ctx, A)
    n = cfg["n"]
    x = np.random.default_rng(9).standard_normal((n, 1))
    LUx = host(hm.hm_matvec(ctx, A, hm.HM_OP_LU, dev(x[:, 0]), F=F))
    Ax_gpu = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, dev(x[:, 0])))
    rows = np.random.default_rng(10).choice(n, 400, replace=False)
    Ax = kernel_matvec_rows(p, A.stats()["h"], rows, x)[:, 0]
    assert np.linalg.norm(Ax_gpu[rows] - Ax) / np.linalg.norm(Ax) < 1e-12
    assert np.linalg.norm(LUx[rows] - Ax) / np.linalg.norm(Ax) <= 10 * cfg["eps"]
