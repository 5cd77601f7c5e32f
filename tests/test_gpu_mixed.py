"""Mixed-precision H-LU (HM_PREC_MIXED) against the FP64 oracles (GPU; calls go through the C ABI).

The factor products of Alg 1 and the rebuild products of the rounded additions run in FP32
(HM_PREC_MIXED), or, for those with at least 128 rows, on the tensor cores with split TF32 and FP32
accumulation (HM_PREC_MIXED_TC); the Gram matrices, truncation core, leaf LU and solves stay FP64. Compared, as every floating-point result here, through reconstructions: the factorization
error ||(A - P L U) X|| / ||A X|| within 10 eps and within 10x the error of the oracle with FP32
products (oracle/mixed.py) on the same matrix, and FP64 iterative refinement reaching a relative
residual of 1e-10 with a forward error below 1e-8 against a dense solve.
"""
import numpy as np
import pytest

import hm_workloads as W
from oracle.geometry import kernel_block
from oracle.hmatrix import HMatrix
from oracle.mixed import MixedHLUFactor

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


def _lu_error(ctx, hm, A, F, n, seed=5):
    X = np.random.default_rng(seed).standard_normal((n, 8))
    Xd = dev(X)
    Ax = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, Xd))
    return fro_ratio(host(hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F)) - Ax, Ax)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("geom,n,eps", [("sphere", 2048, 1e-4), ("cube", 3000, 1e-4), ("cube", 1500, 1e-5)])
def test_mixed_lu_within_ten_eps_and_oracle(ctx, hm, geom, n, eps, prec):
    p = W.points_for(geom, n, 11)
    A = hm.hm_build(ctx, p, 64, 2.0, eps, 64)
    F = hm.hm_lu(ctx, A, precision=prec)
    st = F.stats()
    assert st["precision"] == prec
    assert st["f32_flops"] > 0                      # the FP32 kernel did (some of) the products
    assert (st["tc_flops"] > 0) == (prec == hm.HM_PREC_MIXED_TC)
    err = _lu_error(ctx, hm, A, F, n)
    assert err <= 10 * eps
    F64 = hm.hm_lu(ctx, A)
    err64 = _lu_error(ctx, hm, A, F64, n)
    assert F64.stats()["tc_flops"] == 0 and F64.stats()["f32_flops"] == 0
    assert err <= 3 * err64 + 1e-6                  # the FP32-level products add at most ~1e-6
    if n <= 2048:
        o = MixedHLUFactor(HMatrix(p, 64, 2.0, eps, 64)).factor()
        X = np.random.default_rng(5).standard_normal((n, 8))
        Ao = o.hm.exact_dense()
        oerr = fro_ratio(Ao @ X - o.apply_lu(X), Ao @ X)
        assert oerr <= 10 * eps
        assert err <= 10 * oerr
    # FP64 refinement against the exact kernel wins the accuracy back
    b = np.random.default_rng(6).standard_normal((n, 2))
    x, info = hm.hm_solve(ctx, F, dev(b), A=A, refine_tol=1e-10, max_iter=30, residual_op=hm.HM_OP_EXACT)
    assert info["rel_residual"] <= 1e-10
    xe = np.linalg.solve(kernel_block(p, p, A.stats()["h"]), b)
    assert np.linalg.norm(host(x) - xe) / np.linalg.norm(xe) < 1e-8


def test_mixed_routes_products(ctx, hm):
    """All-dense H-LU (eta = 0): every product has at most one leaf's rows (64), below the
    tensor-core row threshold, so even HM_PREC_MIXED_TC runs them all in FP32: the factor
    reproduces A to the FP32 level (not FP64's 1e-14, not broken). An H-matrix with large
    admissible blocks sends its tall products to the tensor cores under HM_PREC_MIXED_TC only."""
    p = W.cube_surface(700, 3)
    A = hm.hm_build(ctx, p, 64, 0.0, 1e-8, 64)
    F = hm.hm_lu(ctx, A, precision=hm.HM_PREC_MIXED_TC)
    st = F.stats()
    assert st["tc_flops"] == 0 and st["f32_flops"] > 0
    assert 1e-13 < _lu_error(ctx, hm, A, F, 700) < 1e-5
    p2 = W.cube_surface(4000, 3)
    A2 = hm.hm_build(ctx, p2, 64, 2.0, 1e-4, 64)
    for prec in (hm.HM_PREC_MIXED, hm.HM_PREC_MIXED_TC):
        F2 = hm.hm_lu(ctx, A2, precision=prec)
        st = F2.stats()
        assert st["f32_flops"] > 0
        assert (st["tc_flops"] > 0) == (prec == hm.HM_PREC_MIXED_TC)
        assert _lu_error(ctx, hm, A2, F2, 4000) <= 1e-3
        F2.free()


def test_mixed_batch_and_invalid_precision(ctx, hm):
    pts = [W.ellipsoid(n, 7 + n) for n in (900, 1300)]
    mats = [hm.hm_build(ctx, p, 64, 2.0, 1e-4, 64) for p in pts]
    Fs = hm.hm_lu_batch(ctx, mats, precision=hm.HM_PREC_MIXED)
    for A, F, p in zip(mats, Fs, pts):
        assert F.stats()["precision"] == hm.HM_PREC_MIXED
        assert _lu_error(ctx, hm, A, F, p.shape[0]) <= 1e-3
    with pytest.raises(hm.HMError, match="HM_EINVAL"):
        hm.hm_lu(ctx, mats[0], precision=3)
