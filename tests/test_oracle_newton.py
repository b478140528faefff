"""Pins of the oracle's Newton method on power series (Section 2 pseudo code,
with Section 3 test systems and Table 1), against closed-form solutions."""
import os

import numpy as np
import pytest
from fractions import Fraction as Fr

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import exact as ex
from tests import metrics as mt
from tests import systems as ts

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = {2: 1e-28, 4: 1e-58, 8: 1e-118}


@pytest.mark.parametrize("K,d,steps", [(2, 15, 6), (4, 31, 7)])
def test_sqrt_one_plus_t(K, d, steps):
    s, sol, x0 = ts.sqrt_system(K, d)
    x, hist = oracle.newton(s, x0, steps)
    ref = ts.solution_md(sol, K, 1)
    assert np.max(mt.series_rel_error(x, ref)) <= TOL[K]
    # ||f|| falls to the rounding level; the monitor stays at rounding level
    assert hist[-1, 0] < 1e-25 if K == 2 else hist[-1, 0] < 1e-55


@pytest.mark.parametrize("K,C", [(2, 1), (4, 1), (2, 2), (4, 2)])
def test_one_column_exp_solutions(K, C):
    if C == 1:
        alphas = [Fr(-15, 16), Fr(31, 32), Fr(-1)]  # in [-1, -1+delta] u [1-delta, 1], delta = 0.1
    else:
        alphas = [(Fr(3, 5), Fr(4, 5)), (Fr(-4, 5), Fr(3, 5)), (Fr(-1), Fr(0))]  # |alpha| = 1
    d = 15 if K == 2 else 31
    s, sol, x0 = ts.one_column_system(K, C, alphas, d)
    x, _ = oracle.newton(s, x0, 7 if K == 2 else 8)
    assert np.max(mt.series_rel_error(x, ts.solution_md(sol, K, C))) <= TOL[K]


@pytest.mark.parametrize("K,C", [(2, 1), (4, 2)])
def test_two_column_exp_solutions(K, C):
    if C == 1:
        alphas = [Fr(-15, 16), Fr(31, 32), Fr(-1)]
        c1 = [Fr(3, 4), Fr(-5, 4), Fr(1, 2)]
        c2 = [Fr(3, 8), Fr(1), Fr(-5, 8)]
    else:
        alphas = [(Fr(3, 5), Fr(4, 5)), (Fr(-4, 5), Fr(3, 5)), (Fr(-1), Fr(0))]
        c1 = [(Fr(3, 4), Fr(1, 4)), (Fr(-5, 4), Fr(0)), (Fr(1, 2), Fr(-1, 2))]
        c2 = [(Fr(3, 8), Fr(0)), (Fr(1), Fr(1, 8)), (Fr(-5, 8), Fr(1, 4))]
    d = 15 if K == 2 else 31
    s, sol, x0 = ts.two_column_system(K, C, alphas, c1, c2, d)
    x, _ = oracle.newton(s, x0, 7 if K == 2 else 8)
    assert np.max(mt.series_rel_error(x, ts.solution_md(sol, K, C))) <= TOL[K]


def test_table1_inverse_factorials():
    """Newton on x1 = exp(t/16), x1 x2 = exp(17t/16) gives x2 = exp(t): its
    coefficients are the 1/k! of Table 1 (two printed digits).  All terms of
    the series products are positive, so nothing cancels and every coefficient
    keeps its relative precision; with x1 = exp(-t/2) the products cancel by
    a factor 3^k and the high coefficients lose all digits in double double
    (the error growth through the updates described in Section 2)."""
    rows = [line.split() for line in open(os.path.join(GOLDEN, "table1_inverse_factorials.txt"))
            if line.strip() and not line.startswith("#")]
    K, d = 2, 127
    s, sol, x0 = ts.one_column_system(K, 1, [Fr(1, 16), Fr(1)], d, noise=0.0)
    x, _ = oracle.newton(s, x0, 9)
    val = mt.md_value(x)[0, 1]
    for k, printed in rows:
        k, printed = int(k), float(printed)
        assert abs(val[k] - printed) <= 0.05 * printed, (k, val[k], printed)
        exact = Fr(1)
        for j in range(2, k + 1):
            exact /= j
        assert abs(Fr(val[k]) - exact) <= Fr(1, 10 ** 15) * exact
    assert np.max(mt.series_rel_error(x, ts.solution_md(sol, K, 1))) <= 1e-28


PLANTED = [
    wl.small_config(2, 1, n=4, d=7, mono_per_eq=3, kmin=1, kmax=3, steps=6, index=500),
    wl.small_config(4, 1, n=5, d=9, mono_per_eq=3, kmin=2, kmax=4, steps=7, index=501),
    wl.small_config(8, 2, n=3, d=5, mono_per_eq=2, kmin=1, kmax=3, steps=8, index=502),
]


@pytest.mark.parametrize("cfg", PLANTED, ids=lambda c: c.name)
def test_planted_recovery_and_quadratic_convergence(cfg):
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    x = x0
    errs, counts = [], []
    for _ in range(cfg.steps):
        x, _ = oracle.newton(s, x, 1)
        e = mt.series_rel_error(x, xstar)
        errs.append(float(np.max(e[:, 0])))
        counts.append(mt.correct_leading(x, xstar, cfg.tol))
    assert np.max(mt.series_rel_error(x, xstar)) <= cfg.tol
    # the error of x_0 squares from step to step until the rounding floor
    for a, b in zip(errs, errs[1:]):
        if a > 1e3 * cfg.tol:
            assert b <= max(1e4 * a * a, cfg.tol), errs
    # once a coefficient is correct, the count of correct ones at least doubles
    for a, b in zip(counts, counts[1:]):
        if a > 0:
            assert b >= min(2 * a, s.D), counts


def test_converged_update_vanishes():
    """Once x_k is correct, b_k = 0 and so dx_k = 0 (Section 4)."""
    cfg = PLANTED[0]
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    x, _ = oracle.newton(s, x0, cfg.steps)
    x2, hist = oracle.newton(s, x, 1)
    assert hist[0, 2] <= 1e-27 and hist[0, 0] <= 1e-27
    assert np.max(mt.series_rel_error(x2, x)) <= 1e-28


@pytest.mark.parametrize("K,C,D", [(2, 1, 4), (4, 1, 3), (4, 2, 3), (8, 1, 3), (8, 2, 2)])
def test_one_newton_step_exact(K, C, D):
    """One step of the Section 2 pseudo code in exact rationals: f and the
    Jacobian series A_j = [t^j] df/dx at x(t), the block lower triangular
    Toeplitz solve of A dx = -f, and x + dx.  The oracle's step (which
    follows the same steps with its own QR and forward substitution) must
    agree to the md rounding level, with powers among the monomials, a full
    start series (every coefficient nonzero) and the history columns
    ||f(x)||_1 and ||dx||_1 of its leading doubles."""
    n = 3
    # monomial variables; repeated indices are powers
    mons = [(0, [0, 1]), (0, [0, 0, 2]), (0, [0]), (1, [1, 2]), (1, [1]), (1, [2, 2]),
            (2, [2, 0]), (2, [2]), (2, [1, 1, 0])]
    eq = np.array([e for e, _ in mons], dtype=np.int32)
    vptr = np.cumsum([0] + [len(v) for _, v in mons]).astype(np.int32)
    vidx = np.array([q for _, v in mons for q in v], dtype=np.int32)
    M = len(mons)
    coeff = wl.random_md((M, D), K, C, 880 + K + C)
    for m, (e, v) in enumerate(mons):
        if v == [e]:
            coeff[0, 0, m, 0] += 4.0  # a dominant diagonal keeps A_0 well conditioned
    s = wl.System(K, C, n, D - 1, eq, vptr, vidx, coeff, wl.random_md((n, D), K, C, 890 + K))
    x0 = wl.random_md((n, D), K, C, 900 + K + C)

    x1, hist = oracle.newton(s, x0, 1)

    fx = ex.arr_to_fr(x0)
    x = [[fx[i, k] for k in range(D)] for i in range(n)]
    f = ex.system_fr(s, x)
    fc = ex.arr_to_fr(coeff)
    A = [[[ex.zero(C) for _ in range(n)] for _ in range(n)] for _ in range(D)]
    for m, (e, v) in enumerate(mons):
        for q in range(len(v)):  # d/dx_{v[q]}: the product of the other factors
            p = [fc[m, k] for k in range(D)]
            for r, u in enumerate(v):
                if r != q:
                    p = ex.series_mul(p, x[u], D, C)
            for j in range(D):
                A[j][e][v[q]] = ex.add(A[j][e][v[q]], p[j])
    neg_f = [[ex.sub(ex.zero(C), f[i][k]) for k in range(D)] for i in range(n)]
    dx = ex.toeplitz_solve_fr(A, neg_f, C)
    expect = np.empty((n, D), dtype=object)
    for i in range(n):
        for k in range(D):
            expect[i, k] = ex.add(x[i][k], dx[i][k])
    assert ex.worst_rel_log2(x1, expect, floor=1.0) <= -51 * K + 14

    norm_f = sum(ex.absf(f[i][k]) for i in range(n) for k in range(D))
    norm_dx = sum(ex.absf(dx[i][k]) for i in range(n) for k in range(D))
    assert abs(hist[0, 0] - norm_f) <= 1e-13 * norm_f
    assert abs(hist[0, 2] - norm_dx) <= 1e-13 * norm_dx

    # history column 1: the monitor ||b - A dx||_1 of the step (Section 5.4),
    # b = -f and dx the step's computed (rounded) update, both as the md
    # values the oracle holds.  Exactly: the residual of the rounded dx, whose
    # entries are at the md rounding level of the terms A_j dx_{k-j}.
    f_md, A_md = oracle.evaluate(s, x0)
    dx_md = oracle.solve(A_md, -f_md)
    Af, fb, dxf = ex.arr_to_fr(A_md), ex.arr_to_fr(-f_md), ex.arr_to_fr(dx_md)
    norm_r, size = 0.0, 0.0
    for i in range(n):
        for k in range(D):
            r = fb[i, k]
            for j in range(k + 1):
                for l in range(n):
                    r = ex.sub(r, ex.mul(Af[j, i, l], dxf[l, k - j]))
                    size += ex.absf(Af[j, i, l]) * ex.absf(dxf[l, k - j])
            norm_r += ex.absf(r)
    # the oracle rounds each entry once and sums leading doubles
    assert abs(hist[0, 1] - norm_r) <= 1e-12 * norm_r + 2.0 ** (-53 * K) * size
    assert hist[0, 1] <= 2.0 ** (6 - 52 * K) * size


@pytest.mark.parametrize("K,C,n,D", [(2, 1, 3, 4), (4, 2, 2, 3), (8, 1, 2, 3)])
def test_toeplitz_residual_exact(K, C, n, D):
    """The residual r_k = b_k - sum_{j=0..k} A_j dx_{k-j} of Eq. (eqToeplitz)
    for an arbitrary (wrong) dx, entry by entry against exact rationals: a
    dropped j = 0 block, a wrong sign or index, a transposed A_j or a wrong
    norm all fail.  Its 1-norm of leading doubles, and the sampled form over
    a subset of rows scaled by n / rows (Section 5.4)."""
    A = wl.random_md((D, n, n), K, C, 300 + K + C)
    b = wl.random_md((n, D), K, C, 310 + K + C)
    dx = wl.random_md((n, D), K, C, 320 + K + C)
    r, norm = oracle.toeplitz_residual(A, b, dx)
    Af, bf, xf = ex.arr_to_fr(A), ex.arr_to_fr(b), ex.arr_to_fr(dx)
    exact = np.empty((n, D), dtype=object)
    mags = np.zeros((n, D))
    for i in range(n):
        for k in range(D):
            v = bf[i, k]
            for j in range(k + 1):
                for l in range(n):
                    v = ex.sub(v, ex.mul(Af[j, i, l], xf[l, k - j]))
            exact[i, k] = v
            mags[i, k] = ex.absf(v)
    # each entry is its exact value rounded once to K limbs
    assert ex.worst_rel_log2(r, exact) <= 2 - 52 * K
    assert abs(norm - mags.sum()) <= 1e-13 * mags.sum()
    rows = [n - 1]
    _, part = oracle.toeplitz_residual(A, b, dx, rows=rows)
    assert abs(part - n * mags[n - 1].sum()) <= 1e-13 * n * mags[n - 1].sum()
    # the residual of the exact solution is zero up to the md rounding level
    dx_ok = oracle.solve(A, b)
    _, small = oracle.toeplitz_residual(A, b, dx_ok)
    assert small <= 2.0 ** (8 - 52 * K) * (1.0 + norm)
