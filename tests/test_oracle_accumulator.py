"""Pins of the accumulator-based H-LU of the oracle (§2.3, Alg 4-8): the same factors as dense LU
when nothing is compressed, the H-LU accuracy bound with compression and pivoting, fewer
truncations than the recursive H-LU (the point of accumulating), and planted mistakes in the
accumulator bookkeeping that the pins catch."""
import numpy as np
import pytest

import hm_workloads as W
from oracle.accu import AccuHLUFactor
from oracle.geometry import kernel_block
from oracle.hlu import HLUFactor
from oracle.hmatrix import HMatrix, LowRank
from tests.test_oracle_pins import _permute_within_leaf_rows


def _rel(A, f, X):
    return np.linalg.norm(A @ X - f.apply_lu(X)) / np.linalg.norm(A @ X)


def test_accumulator_all_dense_equals_dense_lu():
    p = W.fibonacci_sphere(300, 2)
    hm = HMatrix(p, 64, 0.0, 1e-14, 64)
    f = AccuHLUFactor(hm).factor()
    A = hm.exact_dense()
    assert _rel(A, f, np.eye(hm.n)) < 1e-14
    b = np.random.default_rng(4).standard_normal(hm.n)
    x = f.solve(b)
    assert np.linalg.norm(x - np.linalg.solve(kernel_block(p, p, hm.h), b)) / np.linalg.norm(x) < 1e-12
    assert f.stats.truncations == 0


@pytest.mark.parametrize("eta,eps,tol", [(0.0, 1e-14, 1e-13), (2.0, 1e-12, 1e-10)])
def test_accumulator_with_pivoting(eta, eps, tol):
    p = W.cube_surface(700, 9)
    hm = HMatrix(p, 64, eta, eps, 64)
    pi = _permute_within_leaf_rows(hm, 1)
    f = AccuHLUFactor(hm).factor()
    A = hm.exact_dense()[pi]
    assert _rel(A, f, np.random.default_rng(3).standard_normal((hm.n, 4))) < tol


def test_accumulator_within_ten_eps_and_fewer_truncations():
    p = W.fibonacci_sphere(1024, 11)
    hm = HMatrix(p, 64, 2.0, 1e-4, 64)
    assert any(isinstance(s, LowRank) for s in hm.store.values())
    A = hm.exact_dense()
    fa = AccuHLUFactor(hm).factor()
    err = np.linalg.norm(A - fa.apply_lu(np.eye(hm.n)), 2) / np.linalg.norm(A, 2)
    assert err <= 10 * 1e-4
    fs = HLUFactor(hm).factor()
    assert 0 < fa.stats.truncations < fs.stats.truncations


def test_planted_dropped_pending_update_is_caught(monkeypatch):
    p = W.fibonacci_sphere(1024, 11)
    hm = HMatrix(p, 64, 2.0, 1e-10, 64)
    orig = AccuHLUFactor.shift_upd

    def lossy_shift(self, C):
        self.pending.pop(C.key, None)            # forget the deferred products
        orig(self, C)

    monkeypatch.setattr(AccuHLUFactor, "shift_upd", lossy_shift)
    f = AccuHLUFactor(hm).factor()
    assert _rel(hm.exact_dense(), f, np.random.default_rng(3).standard_normal((hm.n, 2))) > 1e-3


def test_planted_misplaced_restriction_is_caught(monkeypatch):
    """Restricting an accumulator to a son with the son's row offset in place of its column offset
    puts the pieces of off-diagonal sons in the wrong columns."""
    p = W.fibonacci_sphere(1024, 11)
    hm = HMatrix(p, 64, 2.0, 1e-10, 64)

    def swapped_shift(self, C):
        acc = self.acc.pop(C.key, [])
        pend = self.pending.pop(C.key, [])
        for i in range(2):
            for j in range(2):
                Cs = C.sons[i][j]
                ro = Cs.row.lo - C.row.lo
                m, n = Cs.row.size, Cs.col.size
                for (r0, c0, Wp, Zp) in acc:
                    ir0, ir1 = max(r0, ro), min(r0 + Wp.shape[0], ro + m)
                    ic0, ic1 = max(c0, ro), min(c0 + Zp.shape[0], ro + n)
                    if ir0 < ir1 and ic0 < ic1:
                        self.acc.setdefault(Cs.key, []).append(
                            (ir0 - ro, ic0 - ro, Wp[ir0 - r0:ir1 - r0], Zp[ic0 - c0:ic1 - c0]))
                for (alpha, A, B) in pend:
                    for l in range(2):
                        self.add_upd(alpha, A.sons[i][l], B.sons[l][j], Cs)

    monkeypatch.setattr(AccuHLUFactor, "shift_upd", swapped_shift)
    f = AccuHLUFactor(hm).factor()
    assert _rel(hm.exact_dense(), f, np.random.default_rng(3).standard_normal((hm.n, 2))) > 1e-3
