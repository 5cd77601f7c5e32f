"""Python binding of libhmgb300 (H-LU of point-cloud kernel matrices on one GB300).

Argument marshalling only: every call goes through the C ABI declared in
``include/hmgb300.h`` and every step of the computation runs in the library's CUDA
kernels.  PyTorch supplies device memory (the caching allocator, through the allocator
callbacks of the context) and streams.  There is no CPU fallback: if the shared library
has not been built, importing works but the first call raises ``HMError``.

Functions keep the C names (``hm_build``, ``hm_lu``, ``hm_solve``, ``hm_matvec``,
``hm_truncate``, ``hm_structure_build`` ...).  Device vectors are torch tensors in
column-major layout (1-D of length n, or 2-D with stride(0) == 1), in the original point
order.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from .build import LIB, build as _build_lib

__all__ = [
    "HMError", "load_library", "build_library", "HMContext", "HMatrix", "HFactor",
    "hm_ctx_create", "hm_build", "hm_lu", "hm_lu_batch", "hm_solve", "hm_matvec", "hm_truncate", "hm_truncate_noalloc",
    "hm_selftest_reciprocals", "hm_set_gemm_work", "hm_get_gemm_work", "hm_autotune_gemm",
    "hm_set_overlap", "hm_get_overlap",
    "hm_structure_build", "hm_structure_build_accumulator", "hm_structure_build_sparsified",
    "hm_structure_plan_lu_batch", "hm_set_host_threads",
    "header_functions",
    "HM_OP_A", "HM_OP_L", "HM_OP_U", "HM_OP_LU", "HM_OP_EXACT", "HM_PREC_FP64", "HM_PREC_MIXED", "HM_PREC_MIXED_TC",
]

HM_OP_A, HM_OP_L, HM_OP_U, HM_OP_LU, HM_OP_EXACT = 0, 1, 2, 3, 4
HM_PREC_FP64, HM_PREC_MIXED, HM_PREC_MIXED_TC = 0, 1, 2
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hmgb300.h")
ERRORS = {0: "HM_OK", -1: "HM_EINVAL", -2: "HM_ENOMEM", -3: "HM_ECUDA", -4: "HM_ESINGULAR",
          -5: "HM_ETIMEOUT", -6: "HM_ENOTCONV", -7: "HM_EINTERNAL"}
KINDS = ("getrf", "trsm", "gemm", "copy", "stack", "core", "eval", "aca")


class HMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class BuildOpts(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("eta", ctypes.c_double), ("eps", ctypes.c_double),
                ("rank_cap", ctypes.c_int), ("kernel_h", ctypes.c_double), ("prepare_lu", ctypes.c_int)]


class LuOpts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("precision", ctypes.c_int), ("accumulate", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("refine_tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("residual_op", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rel_residual", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nclusters", ctypes.c_int64), ("nleaf_clusters", ctypes.c_int64),
                ("depth", ctypes.c_int64), ("nleaves_dense", ctypes.c_int64),
                ("nleaves_lowrank", ctypes.c_int64), ("value_bytes", ctypes.c_int64), ("h", ctypes.c_double),
                ("eps", ctypes.c_double), ("rank_cap", ctypes.c_int64), ("max_rank", ctypes.c_int64),
                ("sum_rank", ctypes.c_int64), ("dag_nodes", ctypes.c_int64), ("dag_edges", ctypes.c_int64),
                ("dag_levels", ctypes.c_int64), ("dag_seconds", ctypes.c_double),
                ("plan_launches", ctypes.c_int64), ("plan_phases", ctypes.c_int64),
                ("plan_truncations", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64),
                ("plan_seconds", ctypes.c_double), ("seconds", ctypes.c_double),
                ("flops", ctypes.c_double * 5), ("rank_cap_hits", ctypes.c_int64),
                ("singular_pivots", ctypes.c_int64), ("aca_unconverged", ctypes.c_int64),
                ("kind_ms", ctypes.c_double * 8), ("kind_launches", ctypes.c_int64 * 8),
                ("kind_flops", ctypes.c_double * 8), ("launches", ctypes.c_int64),
                ("row_interchanges", ctypes.c_int64), ("precision", ctypes.c_int64), ("tc_ms", ctypes.c_double),
                ("tc_launches", ctypes.c_int64), ("tc_flops", ctypes.c_double), ("f32_ms", ctypes.c_double),
                ("f32_launches", ctypes.c_int64), ("f32_flops", ctypes.c_double),
                ("plan_deferred", ctypes.c_int64), ("accumulate", ctypes.c_int64), ("arena_bytes", ctypes.c_int64),
                ("accumulated_pieces", ctypes.c_int64)]

    def to_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class StructureInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nclusters", ctypes.c_int64), ("nleaves", ctypes.c_int64),
                ("ntasks", ctypes.c_int64), ("nedges", ctypes.c_int64), ("nlevels", ctypes.c_int64),
                ("dag_seconds", ctypes.c_double), ("plan_launches", ctypes.c_int64),
                ("plan_phases", ctypes.c_int64), ("plan_gemm_ops", ctypes.c_int64),
                ("plan_truncations", ctypes.c_int64), ("plan_scratch_bytes", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

_lib = None


def build_library(verbose: bool = False, force: bool = False) -> str:
    return _build_lib(verbose=verbose, force=force)


def header_functions():
    """Names of the functions ``include/hmgb300.h`` declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hm_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def load_library():
    """Load libhmgb300.so (raises HMError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise HMError(-3, f"{LIB} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB)
    P, I, I64, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, None
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "hm_last_error": ([], ctypes.c_char_p),
        "hm_ctx_create": ([I, P, ALLOC_FN, FREE_FN, P, PP], I),
        "hm_ctx_destroy": ([P], V),
        "hm_ctx_set_profiling": ([P, I], I),
        "hm_build": ([P, P, I64, ctypes.POINTER(BuildOpts), PP], I),
        "hm_matrix_free": ([P], V),
        "hm_lu": ([P, P, ctypes.POINTER(LuOpts), PP], I),
        "hm_lu_batch": ([P, P, I, ctypes.POINTER(LuOpts), P], I),
        "hm_factor_free": ([P], V),
        "hm_solve": ([P, P, P, P, P, I64, I64, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)], I),
        "hm_matvec": ([P, P, P, I, D, P, D, P, I64, I64], I),
        "hm_matrix_stats": ([P, ctypes.POINTER(Stats)], I),
        "hm_factor_stats": ([P, ctypes.POINTER(Stats)], I),
        "hm_truncate": ([P, I64, I64, I, P, I64, P, I64, D, I, P, I64, P, I64, ctypes.POINTER(I)], I),
        "hm_truncate_noalloc": ([P, I64, I64, I, P, I64, P, I64, D, I, P, I64, P, I64, ctypes.POINTER(I)], I),
        "hm_selftest_reciprocals": ([P, I, P, P, I64], I),
        "hm_set_gemm_work": ([D], I),
        "hm_get_gemm_work": ([], D),
        "hm_set_overlap": ([I], I),
        "hm_get_overlap": ([], I),
        "hm_autotune_gemm": ([P, P, ctypes.POINTER(LuOpts), P, I, ctypes.POINTER(D), P], I),
        "hm_matrix_layout": ([P, P, P, P, P, P, P], I),
        "hm_matrix_copy_values": ([P, P, P, I], I),
        "hm_structure_build": ([P, I64, I, D, I, PP], I),
        "hm_structure_build_accumulator": ([P, I64, I, D, I, PP], I),
        "hm_structure_build_sparsified": ([P, I64, I, D, I, PP], I),
        "hm_structure_plan": ([P, I, D, I, I, I], I),
        "hm_set_host_threads": ([I], I),
        "hm_structure_plan_lu_batch": ([P, I, D, I], I),
        "hm_structure_plan_table": ([P, I, PP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], I),
        "hm_structure_info_get": ([P, ctypes.POINTER(StructureInfo)], I),
        "hm_structure_export": ([P, P, P, P, P, P, P], I),
        "hm_structure_free": ([P], V),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc, what=""):
    if rc != 0:
        msg = load_library().hm_last_error().decode()
        raise HMError(rc, msg or what)


def _col_major(t, n, name):
    """(pointer, nrhs, ld) of a column-major torch tensor of n rows."""
    if t.dtype.is_floating_point and t.element_size() != 8:
        raise TypeError(f"{name} must be float64")
    if t.dim() == 1:
        if t.shape[0] != n or t.stride(0) != 1:
            raise ValueError(f"{name}: expected a contiguous vector of length {n}")
        return t.data_ptr(), 1, n
    if t.dim() != 2 or t.shape[0] != n or (t.shape[1] > 1 and t.stride(0) != 1):
        raise ValueError(f"{name}: expected an n x nrhs column-major tensor (stride(0) == 1)")
    ld = t.stride(1) if t.shape[1] > 1 else n
    return t.data_ptr(), t.shape[1], ld


# --------------------------------------------------------------------------- thin C-named API
class HMContext:
    """hm_ctx with the PyTorch caching allocator and a torch stream."""

    def __init__(self, device=0, stream=None, torch_allocator=True, admit=None):
        """admit: optional callable(nbytes) -> bool consulted before every device allocation the
        library asks for; False makes the allocator callback return NULL (for tests of the
        HM_ENOMEM paths, or a caller-side memory budget)."""
        import torch
        L = load_library()
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._torch = torch
        if torch_allocator:
            dev, st = self.device, self.stream

            def _alloc(nbytes, user):
                if admit is not None and not admit(int(nbytes)):
                    return None
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:   # out of memory -> NULL -> HM_ENOMEM
                    return None

            def _free(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._af, self._ff = ALLOC_FN(_alloc), FREE_FN(_free)
        else:
            self._af, self._ff = ALLOC_FN(), FREE_FN()
        h = ctypes.c_void_p()
        _check(L.hm_ctx_create(self.device, ctypes.c_void_p(self.stream.cuda_stream), self._af, self._ff, None,
                               ctypes.byref(h)), "hm_ctx_create")
        self.handle = h

    def set_profiling(self, on: bool):
        _check(load_library().hm_ctx_set_profiling(self.handle, int(bool(on))))

    def close(self):
        if self.handle:
            load_library().hm_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hm_ctx_create(device=0, stream=None):
    return HMContext(device, stream)


class HMatrix:
    def __init__(self, ctx, handle, n):
        self.ctx, self.handle, self.n = ctx, handle, n

    def stats(self):
        s = Stats()
        _check(load_library().hm_matrix_stats(self.handle, ctypes.byref(s)))
        return s.to_dict()

    def free(self):
        if self.handle:
            load_library().hm_matrix_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


    def layout(self):
        """Leaf table (nleaves x 10 int64, see hm_matrix_layout), cluster order perm and the
        first position of every cluster."""
        L = load_library()
        nl, nv, nc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(L.hm_matrix_layout(self.handle, None, None, None, ctypes.byref(nl), ctypes.byref(nv),
                                  ctypes.byref(nc)))
        leaves = np.empty((nl.value, 10), dtype=np.int64)
        perm = np.empty(self.n, dtype=np.int64)
        lo = np.empty(nc.value, dtype=np.int64)
        _check(L.hm_matrix_layout(self.handle, leaves.ctypes.data, perm.ctypes.data, lo.ctypes.data, None, None,
                                  None))
        return {"leaves": leaves, "perm": perm, "cluster_lo": lo, "nvalues": nv.value}

    def get_values(self):
        """The block values as a new float64 device tensor."""
        t = self.ctx._torch.empty(self.layout()["nvalues"], dtype=self.ctx._torch.float64,
                                  device=f"cuda:{self.ctx.device}")
        _check(load_library().hm_matrix_copy_values(self.ctx.handle, self.handle, t.data_ptr(), 0))
        return t

    def set_values(self, t):
        """Replace the block values by a float64 device tensor of the same length."""
        if t.dtype != self.ctx._torch.float64 or not t.is_contiguous() or t.numel() != self.layout()["nvalues"]:
            raise ValueError("values: contiguous float64 device tensor of nvalues entries")
        _check(load_library().hm_matrix_copy_values(self.ctx.handle, self.handle, t.data_ptr(), 1))


class HFactor:
    def __init__(self, ctx, handle, A):
        self.ctx, self.handle, self.A = ctx, handle, A

    def stats(self):
        s = Stats()
        _check(load_library().hm_factor_stats(self.handle, ctypes.byref(s)))
        return s.to_dict()

    def free(self):
        if self.handle:
            load_library().hm_factor_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hm_build(ctx, points, leaf_size=64, eta=2.0, eps=1e-6, rank_cap=64, kernel_h=-1.0, prepare_lu=False):
    """H-matrix of a_ij = 1/(4 pi (|x_i - x_j| + h)) for host points (n x 3 float64);
    prepare_lu: plan the H-LU on a host thread while the device assembles the matrix."""
    p = np.ascontiguousarray(points, dtype=np.float64)
    if p.ndim != 2 or p.shape[1] != 3:
        raise ValueError("points must be n x 3")
    o = BuildOpts(int(leaf_size), float(eta), float(eps), int(rank_cap), float(kernel_h), int(bool(prepare_lu)))
    h = ctypes.c_void_p()
    _check(load_library().hm_build(ctx.handle, p.ctypes.data, p.shape[0], ctypes.byref(o), ctypes.byref(h)))
    return HMatrix(ctx, h, p.shape[0])


def hm_lu(ctx, A, eps=0.0, allow_singular=False, precision=0, accumulate=False):
    """H-LU of A (precision: HM_PREC_FP64, HM_PREC_MIXED or HM_PREC_MIXED_TC; accumulate: the
    accumulator H-LU of Alg 4-8)."""
    o = LuOpts(float(eps), int(precision), int(bool(accumulate)))
    h = ctypes.c_void_p()
    rc = load_library().hm_lu(ctx.handle, A.handle, ctypes.byref(o), ctypes.byref(h))
    F = HFactor(ctx, h, A) if h.value else None
    if rc != 0 and not (rc == -4 and allow_singular and F is not None):
        if F is not None:
            F.free()
        _check(rc)
    return F


def hm_lu_batch(ctx, matrices, eps=0.0, allow_singular=False, precision=0, accumulate=False):
    """H-LU of several independent matrices whose waves share kernel launches; one factor each.

    The library sizes its groups of instances by the free device memory; blocks that PyTorch's
    caching allocator holds do not count as free, so they are returned to the driver first."""
    ctx._torch.cuda.empty_cache()
    n = len(matrices)
    hs = (ctypes.c_void_p * n)(*[A.handle for A in matrices])
    outs = (ctypes.c_void_p * n)()
    o = LuOpts(float(eps), int(precision), int(bool(accumulate)))
    rc = load_library().hm_lu_batch(ctx.handle, hs, n, ctypes.byref(o), outs)
    Fs = [HFactor(ctx, ctypes.c_void_p(outs[i]), A) if outs[i] else None for i, A in enumerate(matrices)]
    if rc != 0 and not (rc == -4 and allow_singular and all(F is not None for F in Fs)):
        for F in Fs:
            if F is not None:
                F.free()
        _check(rc)
    return Fs


def hm_solve(ctx, F, b, x=None, A=None, refine_tol=0.0, max_iter=0, residual_op=HM_OP_A):
    """x = (P L U)^{-1} b (device tensors); optional refinement against op(A)."""
    n = F.A.n
    if x is None:
        x = ctx._torch.empty_like(b)
    pb, nb, ldb = _col_major(b, n, "b")
    px, nx, ldx = _col_major(x, n, "x")
    if nb != nx or ldb != ldx:
        raise ValueError("b and x must have the same shape and leading dimension")
    o = SolveOpts(float(refine_tol), int(max_iter), int(residual_op))
    info = SolveInfo()
    _check(load_library().hm_solve(ctx.handle, F.handle, A.handle if A is not None else None, pb, px, nb, ldb,
                                   ctypes.byref(o), ctypes.byref(info)))
    return x, {"iterations": info.iterations, "rel_residual": info.rel_residual}


def hm_matvec(ctx, A, op, x, y=None, alpha=1.0, beta=0.0, F=None):
    n = A.n
    if y is None:
        y = ctx._torch.zeros_like(x)
    px, nx, ldx = _col_major(x, n, "x")
    py, ny, ldy = _col_major(y, n, "y")
    if nx != ny or ldx != ldy:
        raise ValueError("x and y must have the same shape and leading dimension")
    _check(load_library().hm_matvec(ctx.handle, A.handle, F.handle if F is not None else None, int(op),
                                    float(alpha), px, float(beta), py, nx, ldx))
    return y


def hm_truncate(ctx, W, Z, eps, cap=64):
    """Rounded truncation of W Z^T (device tensors, column-major m x K and n x K)."""
    torch = ctx._torch
    m, K = W.shape
    n = Z.shape[0]
    if Z.shape[1] != K:
        raise ValueError("W and Z need the same number of columns")
    Wf = W.t().contiguous().t() if K > 1 else W.contiguous()
    Zf = Z.t().contiguous().t() if K > 1 else Z.contiguous()
    kc = min(cap, m, n)
    U = torch.empty((kc, m), dtype=torch.float64, device=W.device).t()
    V = torch.empty((kc, n), dtype=torch.float64, device=W.device).t()
    k = ctypes.c_int(0)
    _check(load_library().hm_truncate(ctx.handle, m, n, K, Wf.data_ptr(), m, Zf.data_ptr(), n, float(eps), int(cap),
                                      U.data_ptr(), m, V.data_ptr(), n, ctypes.byref(k)))
    return U[:, :k.value], V[:, :k.value]


def hm_truncate_noalloc(W, Z, eps, cap=64, stream=None):
    """hm_truncate without any device allocation inside the library (static scratch).

    For callers that cannot allocate device memory on their call path; the outputs U, V are
    allocated here by the caller side (PyTorch) before the call, the library itself allocates
    nothing. Runs on W's device and the given (or current) torch stream."""
    import torch
    m, K = W.shape
    n = Z.shape[0]
    if Z.shape[1] != K:
        raise ValueError("W and Z need the same number of columns")
    Wf = W.t().contiguous().t() if K > 1 else W.contiguous()
    Zf = Z.t().contiguous().t() if K > 1 else Z.contiguous()
    kc = min(cap, m, n)
    U = torch.empty((kc, m), dtype=torch.float64, device=W.device).t()
    V = torch.empty((kc, n), dtype=torch.float64, device=W.device).t()
    st = stream if stream is not None else torch.cuda.current_stream(W.device)
    k = ctypes.c_int(0)
    with torch.cuda.device(W.device):
        _check(load_library().hm_truncate_noalloc(ctypes.c_void_p(st.cuda_stream), m, n, K, Wf.data_ptr(), m,
                                                  Zf.data_ptr(), n, float(eps), int(cap), U.data_ptr(), m,
                                                  V.data_ptr(), n, ctypes.byref(k)))
    return U[:, :k.value], V[:, :k.value]


def hm_set_gemm_work(fmas_per_cta):
    """GEMM split target (FMAs per CTA, process-wide)."""
    _check(load_library().hm_set_gemm_work(float(fmas_per_cta)))


def hm_get_gemm_work():
    return load_library().hm_get_gemm_work()


def hm_set_overlap(on):
    """Wave overlap of deferred rounded additions on a side stream (process-wide, 0 or 1)."""
    _check(load_library().hm_set_overlap(int(on)))


def hm_get_overlap():
    return load_library().hm_get_overlap()


def hm_autotune_gemm(ctx, A, candidates=(2048.0, 4096.0, 8192.0, 16384.0, 32768.0), eps=0.0, precision=0):
    """Time hm_lu of A at every candidate GEMM split target, keep the fastest set; returns
    (best, {candidate: seconds})."""
    c = (ctypes.c_double * len(candidates))(*[float(v) for v in candidates])
    t = (ctypes.c_double * len(candidates))()
    best = ctypes.c_double()
    o = LuOpts(float(eps), int(precision))
    _check(load_library().hm_autotune_gemm(ctx.handle, A.handle, ctypes.byref(o), c, len(candidates),
                                           ctypes.byref(best), t))
    return best.value, {float(v): t[q] for q, v in enumerate(candidates)}


def hm_selftest_reciprocals(x, which, stream=None):
    """y = f(x) for one of the library's FP64 reciprocal helpers (which: 0 nr_rcp, 1 nr_rsqrt,
    2 fast_rcp, 3 the leaf LU's pivot reciprocal); x a contiguous float64 CUDA tensor."""
    import torch
    if x.dtype != torch.float64 or not x.is_contiguous():
        raise TypeError("x must be a contiguous float64 tensor")
    y = torch.empty_like(x)
    st = stream if stream is not None else torch.cuda.current_stream(x.device)
    with torch.cuda.device(x.device):
        _check(load_library().hm_selftest_reciprocals(ctypes.c_void_p(st.cuda_stream), int(which), x.data_ptr(),
                                                      y.data_ptr(), x.numel()))
    return y


def _dt(fields):
    return np.dtype(fields, align=True)


_U8, _I8, _I4, _F8 = "u8", "i8", "i4", "f8"
# record layouts of the plan tables (the micro-op descriptors of csrc/ops.h)
PLAN_DTYPES = {
    "launches": _dt([("kind", _I4), ("begin", _I4), ("count", _I4), ("gy", _I4), ("gz", _I4), ("first", _I4), ("wave", _I4),
                      ("side", _I4)]),
    "getrf": _dt([("A", _U8), ("piv", _U8), ("b", _I4), ("pad", _I4)]),
    "trsm": _dt([("T", _U8), ("piv", _U8), ("X", _U8), ("x_es", _I8), ("x_vs", _I8), ("nvd", _U8), ("nv", _I4),
                 ("b", _I4), ("mode", _I4), ("pad", _I4)]),
    "gemm": _dt([("A", _U8), ("B", _U8), ("C", _U8), ("a_rs", _I8), ("a_cs", _I8), ("b_rs", _I8), ("b_cs", _I8),
                 ("c_rs", _I8), ("c_cs", _I8), ("md", _U8), ("nd", _U8), ("kd", _U8), ("m", _I4), ("n", _I4),
                 ("k", _I4), ("flags", _I4), ("alpha", _F8), ("fclass", _I4), ("split", _I4)]),
    "copy": _dt([("src", _U8), ("s_rs", _I8), ("s_cs", _I8), ("dst", _U8), ("d_rs", _I8), ("d_cs", _I8),
                 ("md", _U8), ("nd", _U8), ("m", _I4), ("n", _I4), ("mode", _I4), ("pad", _I4), ("alpha", _F8)]),
    "trunc": _dt([("U", _U8), ("V", _U8), ("rank", _U8), ("m", _I4), ("n", _I4), ("cap", _I4), ("Kcap", _I4),
                  ("first_entry", _I4), ("n_entries", _I4), ("Wst", _U8), ("Zst", _U8), ("Gw", _U8), ("Gz", _U8),
                  ("Tw", _U8), ("Tz", _U8), ("work", _U8), ("Kd", _U8), ("eps", _F8), ("flags", _I4),
                  ("pad2", _I4)]),
    "entries": _dt([("W", _U8), ("w_rs", _I8), ("w_cs", _I8), ("Z", _U8), ("z_rs", _I8), ("z_cs", _I8),
                    ("kd", _U8), ("k", _I4), ("row_off", _I4), ("nrows", _I4), ("col_off", _I4), ("ncols", _I4),
                    ("pad", _I4), ("alpha", _F8)]),
    "leaves": _dt([(f, _I8) for f in ("row", "col", "m", "n", "lr", "cap", "off", "voff", "rank_idx",
                                      "piv_off")]),
    "sizes": _dt([(f, _I8) for f in ("scratch_doubles", "scratch_ints", "nvalues", "nranks", "npiv", "ntrunc",
                                     "nwaves", "nphases", "arena_doubles")]),
    "instances": _dt([(f, _I8) for f in ("first_leaf", "nleaves", "base_d", "base_r", "base_p")]),
    "eval": _dt([("D", _U8), ("r0", _I4), ("c0", _I4), ("m", _I4), ("n", _I4)]),
    "aca": _dt([("r0", _I4), ("c0", _I4), ("m", _I4), ("n", _I4), ("U", _U8), ("V", _U8), ("used", _U8),
                ("kd", _U8), ("kmax", _I4), ("pad", _I4), ("tol", _F8)]),
}
PLAN_TABLES = ("launches", "getrf", "trsm", "gemm", "copy", "trunc", "entries", "leaves", "sizes", "instances",
               "eval", "aca")


class Structure:
    """Host-only cluster tree, block tree and H-LU task graph (no GPU needed)."""

    def plan(self, which=0, eps=1e-6, rank_cap=64, nrhs_max=1, threads=0, names=PLAN_TABLES):
        """Host plan (which 0: H-LU at eps, 1: solve for nrhs_max right-hand sides, 2..5: matvec,
        6: assembly, 7: H-LU with wave overlap) as a dict of numpy record arrays, one per table of
        ``PLAN_TABLES`` named in `names`; threads: host threads of the H-LU planner (0: all)."""
        _check(load_library().hm_structure_plan(self.handle, int(which), float(eps), int(rank_cap), int(nrhs_max),
                                                int(threads)))
        return self.plan_tables(names)

    def plan_tables(self, names=PLAN_TABLES):
        """The tables (by name, see ``PLAN_TABLES``) of the structure's last plan."""
        lib = load_library()
        out = {}
        for t, name in enumerate(PLAN_TABLES):
            if name not in names:
                continue
            ptr, cnt, eb = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int64()
            _check(lib.hm_structure_plan_table(self.handle, t, ctypes.byref(ptr), ctypes.byref(cnt), ctypes.byref(eb)))
            dt = PLAN_DTYPES[name]
            if eb.value != dt.itemsize:
                raise HMError(-7, f"plan table {name}: record of {eb.value} bytes, binding expects {dt.itemsize}")
            arr = np.empty(cnt.value, dtype=dt)
            if cnt.value:
                ctypes.memmove(arr.ctypes.data, ptr, cnt.value * eb.value)
            out[name] = arr
        if "sizes" in out:
            out["sizes"] = out["sizes"][0]
        return out

    def __init__(self, handle):
        self.handle = handle
        info = StructureInfo()
        _check(load_library().hm_structure_info_get(handle, ctypes.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in info._fields_}

    def export(self):
        i = self.info
        perm = np.empty(i["n"], dtype=np.int64)
        cl = np.empty((i["nclusters"], 6), dtype=np.int32)
        lv = np.empty((i["nleaves"], 3), dtype=np.int32)
        tasks = np.empty((i["ntasks"], 4), dtype=np.int32)
        edges = np.empty((max(i["nedges"], 1), 2), dtype=np.int32)
        levels = np.empty(i["ntasks"], dtype=np.int32)
        _check(load_library().hm_structure_export(self.handle, perm.ctypes.data, cl.ctypes.data, lv.ctypes.data,
                                                  tasks.ctypes.data, edges.ctypes.data, levels.ctypes.data))
        return dict(perm=perm, clusters=cl, leaves=lv, tasks=tasks, edges=edges[: i["nedges"]], levels=levels)

    def __del__(self):
        try:
            if self.handle:
                load_library().hm_structure_free(self.handle)
                self.handle = None
        except Exception:
            pass


def hm_structure_build_sparsified(points, leaf_size=64, eta=2.0, accumulators=False):
    p = np.ascontiguousarray(points, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load_library().hm_structure_build_sparsified(p.ctypes.data, p.shape[0], int(leaf_size), float(eta),
                                                        int(bool(accumulators)), ctypes.byref(h)))
    return Structure(h)


def hm_structure_build_accumulator(points, leaf_size=64, eta=2.0, merged=False):
    p = np.ascontiguousarray(points, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load_library().hm_structure_build_accumulator(p.ctypes.data, p.shape[0], int(leaf_size), float(eta),
                                                         int(bool(merged)), ctypes.byref(h)))
    return Structure(h)


def hm_set_host_threads(threads=0):
    """Host threads of task-graph construction and planning (0: all hardware threads)."""
    _check(load_library().hm_set_host_threads(int(threads)))


def hm_structure_plan_lu_batch(structures, eps=1e-6, rank_cap=64, names=PLAN_TABLES):
    """One H-LU plan for several independent structures (kept in the first); its tables."""
    arr = (ctypes.c_void_p * len(structures))(*[s.handle for s in structures])
    _check(load_library().hm_structure_plan_lu_batch(arr, len(structures), float(eps), int(rank_cap)))
    return structures[0].plan_tables(names)


def hm_structure_build(points, leaf_size=64, eta=2.0, with_plan=False):
    p = np.ascontiguousarray(points, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load_library().hm_structure_build(p.ctypes.data, p.shape[0], int(leaf_size), float(eta),
                                             int(bool(with_plan)), ctypes.byref(h)))
    return Structure(h)
