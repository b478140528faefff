"""Pins of the oracle's truncated series products and of its evaluation and
differentiation of polynomial systems (Section 5.1 of the paper).

* the paper's worked example of the zero-padded product (golden fixture);
* exact rational convolutions;
* the Speelpenning product prod x_i at x_i(t) = 1 + t, whose value has the
  binomial coefficients of (1+t)^k and whose every partial is (1+t)^(k-1);
* partial derivatives against exact central differences of the system.
"""
import os
from fractions import Fraction as Fr
from math import comb

import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import exact as ex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bound(K, slack=8):
    return -51 * K + np.log2(slack)


def test_padded_product_example_d3():
    rows = [tuple(map(int, line.split())) for line in open(os.path.join(GOLDEN, "series_product_padded_d3.txt"))
            if line.strip() and not line.startswith("#")]
    K, C, D = 4, 1, 3
    a = wl.random_md((D,), K, C, 11)
    b = wl.random_md((D,), K, C, 12)
    fa, fb = ex.arr_to_fr(a), ex.arr_to_fr(b)
    expect = np.empty(D, dtype=object)
    for k in range(D):
        expect[k] = sum((fa[i] * fb[j] for (kk, i, j) in rows if kk == k and j >= 0), Fr(0))
        # the padded form has d terms per coefficient, d = 3
        assert sum(1 for r in rows if r[0] == k) == D
    c = oracle.series_mul(a, b)
    assert ex.worst_rel_log2(c, expect) <= _bound(K)


@pytest.mark.parametrize("K", [1, 2, 4, 8])
@pytest.mark.parametrize("C", [1, 2])
@pytest.mark.parametrize("D", [1, 5, 16])
def test_series_mul_exact(K, C, D):
    a = wl.random_md((D,), K, C, 100 + D)
    b = wl.random_md((D,), K, C, 200 + D)
    fa, fb = ex.arr_to_fr(a), ex.arr_to_fr(b)
    expect = np.empty(D, dtype=object)
    for k, v in enumerate(ex.series_mul(list(fa), list(fb), D, C)):
        expect[k] = v
    c = oracle.series_mul(a, b)
    assert ex.worst_rel_log2(c, expect) <= _bound(K, slack=4 * D)


def _one_monomial_system(K, k, D, n=None, coeff_one=True):
    n = k if n is None else n
    eq = np.zeros(1, np.int32)
    vptr = np.array([0, k], np.int32)
    vidx = np.arange(k, dtype=np.int32)
    coeff = np.zeros((K, 1, 1, D))
    coeff[0, 0, 0, 0] = 1.0
    return wl.System(K, 1, n, D - 1, eq, vptr, vidx, coeff, None)


@pytest.mark.parametrize("K", [2, 4, 8])
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_speelpenning_binomials(K, k):
    D = k + 2
    sysm = _one_monomial_system(K, k, D)
    x = np.zeros((K, 1, k, D))
    x[0, 0, :, 0] = 1.0
    x[0, 0, :, 1] = 1.0  # x_i(t) = 1 + t
    f, A = oracle.evaluate(sysm, x)
    for j in range(D):
        assert f[0, 0, 0, j] == comb(k, j)
        assert np.all(f[1:, 0, 0, j] == 0.0)
        for v in range(k):
            assert A[0, 0, j, 0, v] == comb(k - 1, j)
            assert np.all(A[1:, 0, j, 0, v] == 0.0)


@pytest.mark.parametrize("K", [2, 4])
def test_speelpenning_distinct_factors(K):
    """x_i(t) = 1 + a_i t: d/dx_v of prod x_i is prod_{u != v} (1 + a_u t)."""
    k, D = 4, 6
    a = [Fr(1, 2), Fr(-3, 4), Fr(5, 8), Fr(7, 16)]
    sysm = _one_monomial_system(K, k, D)
    x = np.zeros((K, 1, k, D))
    x[0, 0, :, 0] = 1.0
    x[0, 0, :, 1] = [float(v) for v in a]
    f, A = oracle.evaluate(sysm, x)
    series = [[Fr(1), a[i]] + [Fr(0)] * (D - 2) for i in range(k)]
    for v in range(k):
        p = [Fr(1)] + [Fr(0)] * (D - 1)
        for u in range(k):
            if u != v:
                p = ex.series_mul(p, series[u], D, 1)
        for j in range(D):
            assert ex.md_to_fr(A[:, 0, j, 0, v]) == p[j]


def _exact_series(x):
    fx = ex.arr_to_fr(x)  # [n, D]
    return [list(fx[v]) for v in range(fx.shape[0])]


@pytest.mark.parametrize("K,C", [(2, 1), (4, 1), (4, 2), (8, 2)])
def test_evaluate_small_system_exact(K, C):
    cfg = wl.small_config(K, C, n=4, d=4, mono_per_eq=2, kmin=1, kmax=3, index=300 + K + C)
    sysm, xstar, _ = wl.planted_system(cfg)
    sysm.cst = wl.random_md((sysm.n, sysm.D), K, C, 9)
    x = wl.random_md((sysm.n, sysm.D), K, C, 10)
    f = oracle.evaluate(sysm, x, want_A=False)
    fx = ex.system_fr(sysm, _exact_series(x))
    expect = np.empty((sysm.n, sysm.D), dtype=object)
    for i in range(sysm.n):
        for k in range(sysm.D):
            expect[i, k] = fx[i][k]
    # every entry is a sum of O(1) terms: bound the error against the scale 1
    assert ex.worst_rel_log2(f, expect, floor=1.0) <= _bound(K, slack=64)


@pytest.mark.parametrize("K,C", [(2, 1), (4, 2)])
def test_jacobian_central_differences(K, C):
    """A_j[i][v] = [t^j] df_i/dx_v: exact central differences in the constant
    coefficient of x_v (step h, error O(h^2)) pin the partials independently
    of how the oracle forms them."""
    cfg = wl.small_config(K, C, n=3, d=3, mono_per_eq=2, kmin=1, kmax=3, index=400 + K)
    sysm, _, _ = wl.planted_system(cfg)
    x = wl.random_md((sysm.n, sysm.D), K, C, 20 + K)
    f, A = oracle.evaluate(sysm, x)
    base = _exact_series(x)
    h = Fr(1, 2 ** (60 * K))
    hc = (h, Fr(0)) if C == 2 else h
    expect = np.empty((sysm.D, sysm.n, sysm.n), dtype=object)
    for v in range(sysm.n):
        xp = [list(s) for s in base]
        xm = [list(s) for s in base]
        xp[v][0] = ex.add(xp[v][0], hc)
        xm[v][0] = ex.sub(xm[v][0], hc)
        fp = ex.system_fr(sysm, xp)
        fm = ex.system_fr(sysm, xm)
        for i in range(sysm.n):
            for j in range(sysm.D):
                d = ex.sub(fp[i][j], fm[i][j])
                expect[j, i, v] = (d[0] / (2 * h), d[1] / (2 * h)) if C == 2 else d / (2 * h)
    assert ex.worst_rel_log2(A, expect, floor=1.0) <= _bound(K, slack=64)
