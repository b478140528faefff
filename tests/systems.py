"""Test systems with closed-form power series solutions (test infrastructure).

Right-hand sides are exact rationals (Fractions) rounded to K limbs, so the
expected solutions are known exactly:

* ``sqrt_system``: x1 x2 = 1 + t, x1 - x2 = 0, solved by x1 = x2 = sqrt(1+t)
  with coefficients binom(1/2, k);
* ``one_column_system``: the columns-of-monomials system x^E = b(t) of
  Section 3 with the lower triangular exponent matrix of ones and the
  solutions exp(alpha_k t) (coefficients alpha_k^j / j!);
* ``two_column_system``: c1 x^E1 + c2 x^E2 = b(t) of Section 3 with E1 the
  lower triangular matrix of ones and E2 the matrix of Eq. (equpplow), whose
  row k is row n-k of E1; the same exponential solutions.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np

from paper_2301_12659_gb300 import workloads as wl
from tests import exact as ex


def _series_md(coefs, K, C):
    """Exact series [D] (Fractions or pairs) -> md array [K, C, D]."""
    obj = np.empty(len(coefs), dtype=object)
    for k, v in enumerate(coefs):
        obj[k] = v
    return ex.fr_to_arr(obj, K, C)


def exp_series(alpha, D, C):
    """Coefficients alpha^j / j! of exp(alpha t), exact."""
    out = [ex.one(C)]
    for j in range(1, D):
        term = ex.mul(out[-1], alpha)
        out.append((term[0] / j, term[1] / j) if C == 2 else term / j)
    return out


def _build(K, C, n, D, monomials, cst_exact):
    """monomials: list of (equation, [vars], coefficient Fraction/pair)."""
    eq = np.array([m[0] for m in monomials], np.int32)
    vptr = np.zeros(len(monomials) + 1, np.int32)
    vidx = []
    coeff = np.zeros((K, C, len(monomials), D))
    for q, (i, vs, c) in enumerate(monomials):
        vidx.extend(vs)
        vptr[q + 1] = len(vidx)
        coeff[:, :, q, :] = _series_md([c] + [ex.zero(C)] * (D - 1), K, C)
    cst = np.zeros((K, C, n, D))
    for i in range(n):
        cst[:, :, i, :] = _series_md([ex.sub(ex.zero(C), v) for v in cst_exact[i]], K, C)
    s = wl.System(K, C, n, D - 1, eq, vptr, np.array(vidx, np.int32), coeff, cst)
    s.check()
    return s


def sqrt_system(K, d):
    D = d + 1
    one = Fr(1)
    mons = [(0, [0, 1], one), (1, [0], one), (1, [1], -one)]
    rhs = [[Fr(1), Fr(1)] + [Fr(0)] * (D - 2), [Fr(0)] * D]
    s = _build(K, 1, 2, D, mons, rhs)
    binom = [Fr(1)]
    for k in range(1, D):
        binom.append(binom[-1] * (Fr(1, 2) - (k - 1)) / k)
    sol = np.empty((2, D), dtype=object)
    for v in range(2):
        for k in range(D):
            sol[v, k] = binom[k]
    x0 = np.zeros((K, 1, 2, D))
    x0[0, 0, :, 0] = 1.0
    return s, sol, x0


def _exp_solution(alphas, D, C):
    sol = np.empty((len(alphas), D), dtype=object)
    for v, a in enumerate(alphas):
        for k, c in enumerate(exp_series(a, D, C)):
            sol[v, k] = c
    return sol


def _start(K, C, n, D, noise):
    x0 = np.zeros((K, C, n, D))
    x0[0, 0, :, 0] = 1.0 + noise * np.linspace(-1.0, 1.0, n)
    return x0


def one_column_system(K, C, alphas, d, noise=1e-3):
    """x_1 ... x_i = exp((alpha_1 + ... + alpha_i) t), i = 1..n."""
    n, D = len(alphas), d + 1
    mons, rhs = [], []
    for i in range(n):
        mons.append((i, list(range(i + 1)), ex.one(C)))
        s = ex.zero(C)
        for a in alphas[: i + 1]:
            s = ex.add(s, a)
        rhs.append(exp_series(s, D, C))
    return _build(K, C, n, D, mons, rhs), _exp_solution(alphas, D, C), _start(K, C, n, D, noise)


def two_column_system(K, C, alphas, c1, c2, d, noise=1e-3):
    """c1_i x^{E1_i} + c2_i x^{E2_i} = b_i(t), E1 lower triangular ones,
    row i of E2 = row n-1-i of E1."""
    n, D = len(alphas), d + 1
    mons, rhs = [], []
    for i in range(n):
        e1 = list(range(i + 1))
        e2 = list(range(n - i))
        mons.append((i, e1, c1[i]))
        mons.append((i, e2, c2[i]))
        s1, s2 = ex.zero(C), ex.zero(C)
        for a in [alphas[v] for v in e1]:
            s1 = ex.add(s1, a)
        for a in [alphas[v] for v in e2]:
            s2 = ex.add(s2, a)
        b1, b2 = exp_series(s1, D, C), exp_series(s2, D, C)
        rhs.append([ex.add(ex.mul(c1[i], u), ex.mul(c2[i], w)) for u, w in zip(b1, b2)])
    return _build(K, C, n, D, mons, rhs), _exp_solution(alphas, D, C), _start(K, C, n, D, noise)


def solution_md(sol, K, C):
    return ex.fr_to_arr(sol, K, C)
