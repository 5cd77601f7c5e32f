"""H-matrix storage (Def 2.3), assembly, compression and rounded addition. Oracle; test-only.

Readings (the paper leaves these open):

* Truncation / rounded addition (§2.3 reduces the rank of a sum to a given rank or relative
  accuracy and leaves the method open): for W Z^T, QR-factor both factors
  (Householder, via LAPACK), take the SVD of the small core R_W R_Z^T, keep the
  singular values sigma_i > eps * sigma_1, at most ``rank_cap`` of them (rank 0 if
  sigma_1 = 0).  The result is U = Q_W X_k Sigma_k, V = Q_Z Y_k (V orthonormal).
* Compression of an admissible block: blocks with m*n <= 2^22 are evaluated densely and
  truncated by their SVD; larger blocks use adaptive cross approximation with partial
  pivoting (Bebendorf 2000) to eps/10, followed by the same rounded truncation at eps.
* Storage: an admissible leaf is low-rank U V^T, every other leaf is dense.
"""
from __future__ import annotations

import numpy as np

from .geometry import kernel_block, mean_nn_spacing
from .trees import BlockTree, ClusterTree


class Dense:
    __slots__ = ("D",)

    def __init__(self, D):
        self.D = np.asarray(D, dtype=np.float64)


class LowRank:
    __slots__ = ("U", "V")

    def __init__(self, U, V):
        self.U = np.asarray(U, dtype=np.float64)
        self.V = np.asarray(V, dtype=np.float64)

    @property
    def rank(self) -> int:
        return self.U.shape[1]


class DiagLU:
    """Diagonal leaf after factorization: unit-lower L and upper U packed, LAPACK pivots."""
    __slots__ = ("LU", "piv")

    def __init__(self, LU, piv):
        self.LU = LU
        self.piv = piv


class Stats:
    def __init__(self):
        self.flops = 0.0
        self.cap_hits = 0
        self.truncations = 0
        self.aca_fallbacks = 0


def qr_flops(m: int, k: int) -> float:
    """Householder QR of an m x k matrix: 2 m k^2 - 2 k^3 / 3 (roles swap when k > m)."""
    if m >= k:
        return 2.0 * m * k * k - 2.0 * k ** 3 / 3.0
    return 2.0 * k * m * m - 2.0 * m ** 3 / 3.0


def truncation_flops(m: int, n: int, K: int, k_new: int) -> float:
    """Model flops of one rounded addition with stacked rank K (QR, core, SVD, rebuild)."""
    return (qr_flops(m, K) + qr_flops(n, K) + 2.0 * K ** 3 + 21.0 * K ** 3
            + 2.0 * (m + n) * K * k_new)


def truncate(W: np.ndarray, Z: np.ndarray, eps: float, rank_cap: int, stats: Stats | None = None):
    """Rounded truncation of W Z^T (W: m x K, Z: n x K) to relative accuracy eps, rank <= cap."""
    m, K = W.shape
    n = Z.shape[0]
    if K == 0:
        return np.zeros((m, 0)), np.zeros((n, 0))
    Qw, Rw = np.linalg.qr(W)
    Qz, Rz = np.linalg.qr(Z)
    X, s, Yt = np.linalg.svd(Rw @ Rz.T)
    if s.size == 0 or not s[0] > 0.0:
        k = 0
    else:
        k = int(np.count_nonzero(s > eps * s[0]))
    if k > rank_cap:
        k = rank_cap
        if stats is not None:
            stats.cap_hits += 1
    if stats is not None:
        stats.truncations += 1
        stats.flops += truncation_flops(m, n, K, k)
    U = Qw @ (X[:, :k] * s[:k])
    V = Qz @ Yt[:k].T
    return U, V


def aca(P_rows, P_cols, h, tol, max_rank):
    """Adaptive cross approximation with partial pivoting; returns U (m x k), V (n x k)."""
    m, n = P_rows.shape[0], P_cols.shape[0]
    Us, Vs = [], []
    used = np.zeros(m, dtype=bool)
    i = 0
    norm2 = 0.0
    while len(Us) < max_rank:
        row = kernel_block(P_rows[i:i + 1], P_cols, h)[0]
        for u, v in zip(Us, Vs):
            row = row - u[i] * v
        used[i] = True
        j = int(np.argmax(np.abs(row)))
        if row[j] == 0.0:
            free = np.flatnonzero(~used)
            if free.size == 0:
                break
            i = int(free[0])
            continue
        v = row / row[j]
        u = kernel_block(P_rows, P_cols[j:j + 1], h)[:, 0]
        for uu, vv in zip(Us, Vs):
            u = u - vv[j] * uu
        cross = 0.0
        for uu, vv in zip(Us, Vs):
            cross += (uu @ u) * (vv @ v)
        uu2 = u @ u
        vv2 = v @ v
        norm2 += 2.0 * cross + uu2 * vv2
        Us.append(u)
        Vs.append(v)
        if np.sqrt(uu2 * vv2) <= tol * np.sqrt(abs(norm2)):
            break
        a = np.abs(u)
        a[used] = -1.0
        i = int(np.argmax(a))
        if a[i] < 0.0:
            break
    if not Us:
        return np.zeros((m, 0)), np.zeros((n, 0))
    return np.stack(Us, axis=1), np.stack(Vs, axis=1)


class HMatrix:
    """Kernel matrix a_ij = 1/(4 pi (|x_i - x_j| + h)) stored as an H-matrix in permuted order."""

    def __init__(self, points, leaf_size=64, eta=2.0, eps=1e-6, rank_cap=64, h=None,
                 dense_svd_limit=1 << 22):
        self.points = np.asarray(points, dtype=np.float64)
        self.n = self.points.shape[0]
        self.ct = ClusterTree(self.points, leaf_size)
        self.bt = BlockTree(self.ct, eta)
        self.h = mean_nn_spacing(self.points) if h is None else float(h)
        self.eps = float(eps)
        self.rank_cap = int(rank_cap)
        self.stats = Stats()
        P = self.points[self.ct.perm]
        self.P = P
        self.store = {}
        for b in self.bt.leaves():
            rows = P[b.row.lo:b.row.hi]
            cols = P[b.col.lo:b.col.hi]
            if b.adm:
                m, n = rows.shape[0], cols.shape[0]
                if m * n <= dense_svd_limit:
                    D = kernel_block(rows, cols, self.h)
                    U, s, Vt = np.linalg.svd(D, full_matrices=False)
                    if s.size and s[0] > 0.0:
                        k = min(int(np.count_nonzero(s > self.eps * s[0])), self.rank_cap)
                    else:
                        k = 0
                    self.store[b.key] = LowRank(U[:, :k] * s[:k], Vt[:k].T)
                else:
                    self.stats.aca_fallbacks += 1
                    U0, V0 = aca(rows, cols, self.h, self.eps / 10.0, 4 * self.rank_cap)
                    U, V = truncate(U0, V0, self.eps, self.rank_cap)
                    self.store[b.key] = LowRank(U, V)
            else:
                self.store[b.key] = Dense(kernel_block(rows, cols, self.h))

    # -- dense views (tiny n only) --------------------------------------------------------
    def to_dense(self, store=None) -> np.ndarray:
        store = self.store if store is None else store
        A = np.zeros((self.n, self.n))
        for b in self.bt.leaves():
            A[b.row.lo:b.row.hi, b.col.lo:b.col.hi] = leaf_dense(store[b.key])
        return A

    def exact_dense(self) -> np.ndarray:
        """Exact kernel matrix in permuted order."""
        return kernel_block(self.P, self.P, self.h)

    def ranks(self):
        return [s.rank for s in self.store.values() if isinstance(s, LowRank)]


def leaf_dense(s) -> np.ndarray:
    if isinstance(s, Dense):
        return s.D
    if isinstance(s, LowRank):
        return s.U @ s.V.T
    raise TypeError("factored diagonal leaf has no single dense value")


def block_matvec(bt, store, blk, X, stats=None, transpose=False):
    """Y = M_blk X (or M_blk^T X) for the H-matrix block ``blk`` and a thin dense X."""
    t, s = blk.row, blk.col
    if transpose:
        Y = np.zeros((s.size, X.shape[1]))
    else:
        Y = np.zeros((t.size, X.shape[1]))
    for lf in bt.leaves_under(blk):
        st = store[lf.key]
        r0, r1 = lf.row.lo - t.lo, lf.row.hi - t.lo
        c0, c1 = lf.col.lo - s.lo, lf.col.hi - s.lo
        r = X.shape[1]
        if isinstance(st, Dense):
            if transpose:
                Y[c0:c1] += st.D.T @ X[r0:r1]
            else:
                Y[r0:r1] += st.D @ X[c0:c1]
            if stats is not None:
                stats.flops += 2.0 * st.D.shape[0] * st.D.shape[1] * r
        elif isinstance(st, LowRank):
            k = st.rank
            if transpose:
                Y[c0:c1] += st.V @ (st.U.T @ X[r0:r1])
            else:
                Y[r0:r1] += st.U @ (st.V.T @ X[c0:c1])
            if stats is not None:
                stats.flops += 2.0 * k * r * (st.U.shape[0] + st.V.shape[0])
        else:
            raise TypeError("block_matvec reached a factored diagonal leaf")
    return Y
