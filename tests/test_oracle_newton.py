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
