"""Pins of the oracle's linear algebra: Householder QR of A0 (Section 5.3)
and the solution of the block lower triangular Toeplitz system of
Eq. (eqToeplitz) (Section 2), against exact rational arithmetic."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import exact as ex


def _dominant(n, K, C, seed):
    A0 = wl.random_md((n, n), K, C, seed)
    for i in range(n):
        A0[0, 0, i, i] += n  # keep the exact problem well conditioned
    return A0


@pytest.mark.parametrize("K", [2, 4, 8])
@pytest.mark.parametrize("C", [1, 2])
@pytest.mark.parametrize("n", [1, 3, 5])
def test_qr_invariants(K, C, n):
    A0 = wl.random_md((n, n), K, C, 50 + n)  # no dominance needed: full rank a.s.
    Q, R = oracle.qr(A0)
    fA, fQ, fR = ex.arr_to_fr(A0), ex.arr_to_fr(Q), ex.arr_to_fr(R)
    bound = Fr(64 * n) * Fr(2) ** (-51 * K)
    for i in range(n):
        for j in range(i):
            assert ex.absq(fR[i, j]) == 0
    for i in range(n):
        for j in range(n):
            qhq = ex.zero(C)
            qr_ = ex.zero(C)
            for k in range(n):
                qhq = ex.add(qhq, ex.mul(ex.conj(fQ[k, i]), fQ[k, j]))
                qr_ = ex.add(qr_, ex.mul(fQ[i, k], fR[k, j]))
            eye = ex.one(C) if i == j else ex.zero(C)
            assert ex.absq(ex.sub(qhq, eye)) <= bound ** 2
            assert ex.absq(ex.sub(qr_, fA[i, j])) <= (bound * n) ** 2


def test_qr_zero_column_is_singular():
    A0 = wl.random_md((3, 3), 2, 1, 7)
    A0[:, :, :, 1] = 0.0
    with pytest.raises(oracle.OracleError):
        oracle.qr(A0)


@pytest.mark.parametrize("K,C,n,D", [(2, 1, 3, 4), (4, 1, 2, 5), (4, 2, 3, 3), (8, 1, 2, 3), (8, 2, 2, 2)])
def test_block_toeplitz_solve_exact(K, C, n, D):
    A = wl.random_md((D, n, n), K, C, 60 + K + C + n)
    for i in range(n):
        A[0, 0, 0, i, i] += n
    b = wl.random_md((n, D), K, C, 70 + K)
    dx = oracle.solve(A, b)
    fA, fb = ex.arr_to_fr(A), ex.arr_to_fr(b)
    Al = [[[fA[j, i, l] for l in range(n)] for i in range(n)] for j in range(D)]
    bl = [[fb[i, k] for k in range(D)] for i in range(n)]
    sol = ex.toeplitz_solve_fr(Al, bl, C)
    expect = np.empty((n, D), dtype=object)
    for i in range(n):
        for k in range(D):
            expect[i, k] = sol[i][k]
    # errors propagate through the right hand side updates (Section 2), so the
    # bound grows with the coefficient index; scale floor 1 for tiny entries
    assert ex.worst_rel_log2(dx, expect, floor=1.0) <= -51 * K + 12


def test_solve_recovers_known_solution_structure():
    """b = T x for a chosen x: the solve returns x (D = 1 reduces to A0 x = b)."""
    K, C, n = 4, 1, 4
    A = _dominant(n, K, C, 3)[:, :, None]
    x = wl.random_md((n, 1), K, C, 4)
    fA, fx = ex.arr_to_fr(A), ex.arr_to_fr(x)
    bobj = np.empty((n, 1), dtype=object)
    for i in range(n):
        acc = Fr(0)
        for l in range(n):
            acc += fA[0, i, l] * fx[l, 0]
        bobj[i, 0] = acc
    b = ex.fr_to_arr(bobj, K, C)
    dx = oracle.solve(A, b)
    assert ex.worst_rel_log2(dx, fx, floor=1.0) <= -51 * K + 10
