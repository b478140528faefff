"""Pins of the oracle's stated-accuracy variant of the forward substitution:
stages k >= first_stage form their right hand side updates
sum_{j>=1} A_j dx_{k-j} (Section 5.4) in K/2 limbs, everything else in K
limbs.  Pinned against the plain method (bitwise on the early stages, within
the K/2-limb rounding level on the late ones) and against a planted series
solution that Newton must still recover to the full K-limb tolerance, since
f(x(t)) and the residuals stay in K limbs."""
import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import metrics as mt


def _problem(K, C, n, D, seed):
    A = wl.random_md((D, n, n), K, C, seed)
    for i in range(n):
        A[0, 0, 0, i, i] += n
    b = wl.random_md((n, D), K, C, seed + 1)
    return A, b


@pytest.mark.parametrize("K,C", [(2, 1), (4, 1), (8, 1), (8, 2)])
def test_late_variant_against_plain(K, C):
    n, D, late = 4, 12, 6
    A, b = _problem(K, C, n, D, 70 + K + C)
    plain = oracle.solve(A, b)
    var = oracle.solve(A, b, late=(late, K // 2))
    # stages before the first late one are the plain method, bit for bit
    assert np.array_equal(var[..., :late], plain[..., :late])
    err = mt.series_rel_error(var, plain)[:, late:]
    eps_half = 2.0 ** (-52 * (K // 2))
    # the late stages carry K/2-limb rounding of the updates: bounded by a
    # modest multiple of its unit roundoff, and really present
    assert err.max() <= 1e4 * eps_half, err.max()
    assert err.max() >= 1e-6 * eps_half, err.max()


@pytest.mark.parametrize("K", [2, 8])
def test_late_variant_off_is_plain(K):
    n, D = 3, 8
    A, b = _problem(K, 1, n, D, 90 + K)
    plain = oracle.solve(A, b)
    assert np.array_equal(oracle.solve(A, b, late=(D, K // 2)), plain)   # no late stage
    assert np.array_equal(oracle.solve(A, b, late=(1, K)), plain)        # full limbs


@pytest.mark.parametrize("K,C", [(8, 2), (4, 1)])
def test_newton_with_late_updates_recovers_plant(K, C):
    """Residuals stay in K limbs, so Newton corrects the K/2-limb updates and
    still reaches the K-limb tolerance on the planted solution."""
    cfg = wl.small_config(K, C, n=3, d=11, mono_per_eq=2, kmin=1, kmax=3, steps=9, index=505)
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    x, hist = oracle.newton(s, x0, cfg.steps, late=(6, K // 2))
    assert np.max(mt.series_rel_error(x, xstar)) <= cfg.tol
    # and the variant's first step differs from the plain one only at the
    # K/2-limb level on the late coefficients
    x1p, _ = oracle.newton(s, x0, 1)
    x1v, _ = oracle.newton(s, x0, 1, late=(6, K // 2))
    assert np.array_equal(x1v[..., :6], x1p[..., :6])
    assert np.max(mt.series_rel_error(x1v, x1p)) <= 1e4 * 2.0 ** (-52 * (K // 2))
