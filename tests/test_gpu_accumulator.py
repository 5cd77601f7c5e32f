"""The accumulator H-LU on the GPU (§2.3, Alg 4-8; hm_lu_opts.accumulate = 1).

The update pieces of every low-rank leaf are collected and added in one rounded addition
before the leaf is used. Compared with the oracle's accumulator H-LU (``oracle/accu.py``,
piece lists) on the same points: both within 10 eps of the exact kernel, the GPU's error
within 10x the oracle's; fewer rounded additions than the H-LU of Alg 2; the same factors
(within the tolerance of the factorization) with and without the wave overlap; refinement
against the exact kernel reaches the dense solution.
"""
import numpy as np
import pytest

import hm_workloads as W
from oracle.accu import AccuHLUFactor
from oracle.geometry import kernel_block
from oracle.hmatrix import HMatrix

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


@pytest.mark.parametrize("geom,n,eps", [("sphere", 2048, 1e-4), ("cube", 2048, 1e-6), ("sphere", 1024, 1e-8)])
def test_accumulator_lu_against_oracle(ctx, hm, geom, n, eps):
    p = W.points_for(geom, n, 11)
    A = hm.hm_build(ctx, p, 64, 2.0, eps, 64)
    F0 = hm.hm_lu(ctx, A)
    trunc0 = F0.stats()["plan_truncations"]
    F0.free()
    F = hm.hm_lu(ctx, A, accumulate=True)
    st = F.stats()
    assert st["accumulate"] == 1 and st["singular_pivots"] == 0
    assert st["arena_bytes"] > 0 and st["accumulated_pieces"] > 0
    assert st["plan_truncations"] < trunc0
    X = np.random.default_rng(5).standard_normal((n, 8))
    Xd = dev(X)
    Ax = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, Xd))
    err = fro_ratio(host(hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F)) - Ax, Ax)
    assert err <= 10 * eps
    o = AccuHLUFactor(HMatrix(p, 64, 2.0, eps, 64)).factor()
    Ao = o.hm.exact_dense()
    oerr = fro_ratio(Ao @ X - o.apply_lu(X), Ao @ X)
    assert oerr <= 10 * eps
    assert err <= 10 * max(oerr, 1e-15)
    b = np.random.default_rng(6).standard_normal((n, 2))
    x, info = hm.hm_solve(ctx, F, dev(b), A=A, refine_tol=1e-10, max_iter=30, residual_op=hm.HM_OP_EXACT)
    assert info["rel_residual"] <= 1e-10
    xe = np.linalg.solve(kernel_block(p, p, A.stats()["h"]), b)
    assert np.linalg.norm(host(x) - xe) / np.linalg.norm(xe) < 1e-8
    F.free()
    A.free()


def test_accumulator_with_and_without_overlap(ctx, hm):
    n, eps = 8192, 1e-6
    A = hm.hm_build(ctx, W.cube_surface(n, 31), 64, 2.0, eps, 64)
    X = np.random.default_rng(7).standard_normal((n, 4))
    Xd = dev(X)
    Ax = host(hm.hm_matvec(ctx, A, hm.HM_OP_EXACT, Xd))
    before = hm.hm_get_overlap()
    out = {}
    try:
        for on in (1, 0):
            hm.hm_set_overlap(on)
            F = hm.hm_lu(ctx, A, accumulate=True)
            st = F.stats()
            assert (st["plan_deferred"] > 0) == (on == 1)
            out[on] = host(hm.hm_matvec(ctx, A, hm.HM_OP_LU, Xd, F=F))
            assert fro_ratio(out[on] - Ax, Ax) <= 10 * eps
            F.free()
    finally:
        hm.hm_set_overlap(before)
    assert fro_ratio(out[1] - out[0], Ax) <= eps
    with pytest.raises(hm.HMError, match="HM_EINVAL"):
        hm.hm_lu_batch(ctx, [A], accumulate=True)
    A.free()
