"""The allocation-free rounded truncation, checked against hm_truncate (GPU).

hm_truncate_noalloc serves callers that cannot allocate device memory on their call path
(fixed device budgets sized at start-up, plugins inside another framework's memory pool).
It must give the same truncation as hm_truncate -- same rank, same product within the
tolerance of the truncation tests -- on consecutive calls that share its static scratch,
and must not allocate (PyTorch's allocator sees no change across the call).  This file is
collected last so that a stop at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_07531_gb300 as hm
    hm.build_library()
    return hm


def _case(m, n, r, K, seed):
    rng = np.random.default_rng(seed)
    s = np.logspace(0, -12.37, r)
    Q1, _ = np.linalg.qr(rng.standard_normal((m, r)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, r)))
    Qm, _ = np.linalg.qr(rng.standard_normal((r, r)))
    Mx = Qm @ np.diag(np.logspace(0, 1, r))
    Wm = np.hstack([(Q1 * s) @ Mx, np.zeros((m, K - r))])
    Zm = np.hstack([Q2 @ np.linalg.inv(Mx).T, rng.standard_normal((n, K - r))])
    exact = Q1 @ np.diag(s) @ Q2.T
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()
    return dev(Wm), dev(Zm), exact, s


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_noalloc_matches_hm_truncate_on_consecutive_calls(hm, eps):
    ctx = hm.HMContext(0)
    cases = [(700, 513, 30, 40, 1), (300, 90, 20, 24, 2)]   # the second call is smaller
    for m, n, r, K, seed in cases:
        Wd, Zd, exact, s = _case(m, n, r, K, seed)
        U1, V1 = hm.hm_truncate(ctx, Wd, Zd, eps, 64)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        kc = min(64, m, n)
        U2 = torch.empty((kc, m), dtype=torch.float64, device="cuda").t()
        V2 = torch.empty((kc, n), dtype=torch.float64, device="cuda").t()
        grown = torch.cuda.memory_allocated() - before
        import ctypes
        k = ctypes.c_int(0)
        st = torch.cuda.current_stream()
        rc = hm.load_library().hm_truncate_noalloc(ctypes.c_void_p(st.cuda_stream), m, n, K, Wd.data_ptr(), m,
                                                   Zd.data_ptr(), n, eps, 64, U2.data_ptr(), m, V2.data_ptr(), n,
                                                   ctypes.byref(k))
        assert rc == 0, hm.load_library().hm_last_error()
        assert torch.cuda.memory_allocated() - before == grown   # nothing allocated by the call
        assert k.value == U1.shape[1]
        k_ref = int(np.count_nonzero(s > eps * s[0]))
        assert k.value == k_ref
        P1 = (U1 @ V1.t()).cpu().numpy()
        P2 = (U2[:, :k.value] @ V2[:, :k.value].t()).cpu().numpy()
        tail = s[k_ref] if k_ref < r else 0.0
        assert np.linalg.norm(P2 - exact, 2) <= tail + 1e-7 * s[0]
        # same bound as the truncation tests: the Gram reduction adds in a nondeterministic
        # order, so two calls agree to the truncation's accuracy floor (1e-7 sigma_1), not bitwise
        assert np.linalg.norm(P2 - P1, 2) <= 1e-7 * s[0]
        # the Python wrapper of the same entry point agrees as well
        U3, V3 = hm.hm_truncate_noalloc(Wd, Zd, eps, 64)
        assert np.linalg.norm((U3 @ V3.t()).cpu().numpy() - P1, 2) <= 1e-7 * s[0]


def test_noalloc_rejects_sizes_beyond_its_scratch(hm):
    W = torch.zeros((8000, 130), dtype=torch.float64, device="cuda")
    Z = torch.zeros((8000, 130), dtype=torch.float64, device="cuda")
    with pytest.raises(hm.HMError, match="static scratch"):
        hm.hm_truncate_noalloc(W, Z, 1e-6, 64)


def test_noalloc_writes_strided_outputs(hm):
    """U and V written with leading dimensions larger than their row counts (column slices of
    bigger buffers): the padding rows keep their values and the product matches hm_truncate."""
    import ctypes
    ctx = hm.HMContext(0)
    m, n, r, K, eps = 300, 200, 20, 24, 1e-6
    Wd, Zd, exact, s = _case(m, n, r, K, 5)
    U1, V1 = hm.hm_truncate(ctx, Wd, Zd, eps, 64)
    ldu, ldv = m + 13, n + 7
    kc = min(64, m, n)
    Ub = torch.full((kc, ldu), 7.0, dtype=torch.float64, device="cuda")   # column-major ldu x kc
    Vb = torch.full((kc, ldv), -3.0, dtype=torch.float64, device="cuda")
    k = ctypes.c_int(0)
    st = torch.cuda.current_stream()
    rc = hm.load_library().hm_truncate_noalloc(ctypes.c_void_p(st.cuda_stream), m, n, K, Wd.data_ptr(), m,
                                               Zd.data_ptr(), n, eps, 64, Ub.data_ptr(), ldu, Vb.data_ptr(), ldv,
                                               ctypes.byref(k))
    assert rc == 0, hm.load_library().hm_last_error()
    kk = k.value
    assert kk == U1.shape[1]
    Ubh, Vbh = Ub.cpu().numpy(), Vb.cpu().numpy()
    assert (Ubh[:kk, m:] == 7.0).all() and (Vbh[:kk, n:] == -3.0).all()   # padding rows untouched
    assert (Ubh[kk:] == 7.0).all() and (Vbh[kk:] == -3.0).all()           # columns past the rank
    P2 = Ubh[:kk, :m].T @ Vbh[:kk, :n]
    P1 = (U1 @ V1.t()).cpu().numpy()
    assert np.linalg.norm(P2 - P1, 2) <= 1e-7 * s[0]
