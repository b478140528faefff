"""Exact rational arithmetic helpers for the pins (test infrastructure).

Doubles are dyadic rationals, so a multiple double value (a sum of limbs) is
an exact ``fractions.Fraction``.  Complex values are (re, im) pairs of
Fractions.  Nothing here implements the multiple double algorithms; it only
converts between md arrays and exact rationals and does exact polynomial and
linear algebra on small cases.
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np


def md_to_fr(limbs) -> Fr:
    return sum((Fr(float(v)) for v in limbs), Fr(0))


def fr_to_md(r: Fr, K: int) -> list:
    """K limbs: each the double nearest the remaining exact value."""
    out = []
    for _ in range(K):
        v = float(r)
        out.append(v)
        r -= Fr(v)
    return out


def arr_to_fr(a: np.ndarray):
    """[K, C, *S] float64 -> object array [*S] of Fractions (C=1) or (re, im) tuples."""
    K, C = a.shape[:2]
    shape = a.shape[2:]
    out = np.empty(shape, dtype=object)
    for idx in np.ndindex(*shape):
        re = md_to_fr(a[(slice(None), 0) + idx])
        if C == 1:
            out[idx] = re
        else:
            out[idx] = (re, md_to_fr(a[(slice(None), 1) + idx]))
    return out


def fr_to_arr(obj: np.ndarray, K: int, C: int) -> np.ndarray:
    shape = obj.shape
    a = np.zeros((K, C) + shape)
    for idx in np.ndindex(*shape):
        v = obj[idx]
        if C == 1:
            a[(slice(None), 0) + idx] = fr_to_md(v, K)
        else:
            a[(slice(None), 0) + idx] = fr_to_md(v[0], K)
            a[(slice(None), 1) + idx] = fr_to_md(v[1], K)
    return a


# ---- scalar ops that work on Fractions and (re, im) pairs -------------------

def add(a, b):
    if isinstance(a, tuple):
        return (a[0] + b[0], a[1] + b[1])
    return a + b


def sub(a, b):
    if isinstance(a, tuple):
        return (a[0] - b[0], a[1] - b[1])
    return a - b


def mul(a, b):
    if isinstance(a, tuple):
        return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])
    return a * b


def div(a, b):
    if isinstance(a, tuple):
        den = b[0] * b[0] + b[1] * b[1]
        return ((a[0] * b[0] + a[1] * b[1]) / den, (a[1] * b[0] - a[0] * b[1]) / den)
    return a / b


def conj(a):
    return (a[0], -a[1]) if isinstance(a, tuple) else a


def zero(C):
    return (Fr(0), Fr(0)) if C == 2 else Fr(0)


def one(C):
    return (Fr(1), Fr(0)) if C == 2 else Fr(1)


def absq(a) -> Fr:
    """|a|^2 exactly."""
    if isinstance(a, tuple):
        return a[0] * a[0] + a[1] * a[1]
    return a * a


def absf(a) -> float:
    return float(absq(a)) ** 0.5


# ---- series ------------------------------------------------------------------

def series_mul(a, b, D, C):
    out = []
    for k in range(D):
        acc = zero(C)
        for i in range(k + 1):
            acc = add(acc, mul(a[i], b[k - i]))
        out.append(acc)
    return out


def system_fr(sysm, x):
    """Exact f(x(t)) [n][D] for a workloads.System and exact series x [n][D]."""
    C, n, D = sysm.C, sysm.n, sysm.D
    coeff = arr_to_fr(sysm.coeff)
    cst = arr_to_fr(sysm.cst) if sysm.cst is not None else None
    f = [[zero(C) if cst is None else cst[i, k] for k in range(D)] for i in range(n)]
    for m in range(sysm.M):
        i = int(sysm.eq[m])
        p = [coeff[m, k] for k in range(D)]
        for v in sysm.vidx[sysm.vptr[m]:sysm.vptr[m + 1]]:
            p = series_mul(p, x[int(v)], D, C)
        for k in range(D):
            f[i][k] = add(f[i][k], p[k])
    return f


# ---- exact linear algebra ------------------------------------------------------

def solve_dense(Amat, b, C):
    """Gaussian elimination with exact rationals (partial pivoting on nonzero)."""
    N = len(b)
    M = [list(Amat[i]) + [b[i]] for i in range(N)]
    for col in range(N):
        piv = next(r for r in range(col, N) if absq(M[r][col]) != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(N):
            if r != col and absq(M[r][col]) != 0:
                fac = div(M[r][col], M[col][col])
                M[r] = [sub(M[r][c], mul(fac, M[col][c])) for c in range(N + 1)]
    return [div(M[i][N], M[i][i]) for i in range(N)]


def toeplitz_solve_fr(A, b, C):
    """Exact solution of sum_{j<=k} A_j x_{k-j} = b_k; A [D][n][n], b [n][D]."""
    D, n = len(A), len(A[0])
    N = n * D
    T = [[zero(C) for _ in range(N)] for _ in range(N)]
    rhs = [zero(C)] * N
    for k in range(D):
        for i in range(n):
            rhs[k * n + i] = b[i][k]
            for j in range(k + 1):
                for l in range(n):
                    T[k * n + i][(k - j) * n + l] = A[j][i][l]
    sol = solve_dense(T, rhs, C)
    return [[sol[k * n + i] for k in range(D)] for i in range(n)]


def _log2(q: Fr) -> float:
    if q == 0:
        return float("-inf")
    return math.log2(q.numerator) - math.log2(q.denominator)


def worst_rel_log2(got: np.ndarray, exact: np.ndarray, floor=None) -> float:
    """log2 of max |got - exact| / max(|exact|, floor) over the entries (exact
    given as an object array of Fractions or (re, im) pairs); -inf if exact."""
    g = arr_to_fr(got)
    worst = float("-inf")
    for idx in np.ndindex(*exact.shape):
        e = exact[idx]
        err = absq(sub(g[idx], e))
        den = absq(e)
        if floor is not None:
            den = max(den, Fr(floor) ** 2)
        if den == 0:
            if err != 0:
                return float("inf")
            continue
        worst = max(worst, 0.5 * _log2(err / den))
    return worst
