"""Pins of the oracle's multiple double primitives against exact rationals.

Multiple double numbers are unevaluated sums of nonoverlapping doubles
(Section 1.2 of the paper).  The oracle rounds the exact result of every
operation once, so |r - exact| <= 2^(-51 K) |exact| (K limbs).  Inputs are
dyadic rationals, so the exact result of +, -, * is a Fraction; division is
checked through a/b exactly and the square root through r^2 = a.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import exact as ex

KS = [1, 2, 4, 8]


def _random_pair(K, C, N, seed):
    a = wl.random_md((N,), K, C, seed)
    b = wl.random_md((N,), K, C, seed + 1)
    # scale some entries far apart and plant cancellations (adversarial cases)
    scale = 2.0 ** np.round(40 * wl.uniform_pm1(seed + 2, N))
    a[:, :, : N // 4] *= scale[: N // 4]
    b[:, :, N // 4: N // 2] = -a[:, :, N // 4: N // 2]            # exact cancellation
    b[-1, :, N // 4: N // 2] += 2.0 ** -300                        # ... up to a tiny remainder
    b[:, :, N // 2: N // 2 + 2] = 0.0                             # zero operand
    return a, b


def _bound_ok(got, exactv, K, slack=1):
    """|got - exact| <= slack * 2^(-51K) |exact| for every entry."""
    bound = Fr(slack) * Fr(2) ** (-51 * K)
    g = ex.arr_to_fr(got)
    for idx in np.ndindex(*exactv.shape):
        err = ex.absq(ex.sub(g[idx], exactv[idx]))
        if err > bound * bound * ex.absq(exactv[idx]):
            return False, idx
    return True, None


@pytest.mark.parametrize("K", KS)
@pytest.mark.parametrize("C", [1, 2])
@pytest.mark.parametrize("op", ["add", "sub", "mul"])
def test_md_ring_ops_exact_rounding(K, C, op):
    N = 40
    a, b = _random_pair(K, C, N, 1000 + 10 * K + C)
    r = oracle.md_binary(op, a, b)
    fa, fb = ex.arr_to_fr(a), ex.arr_to_fr(b)
    fn = {"add": ex.add, "sub": ex.sub, "mul": ex.mul}[op]
    exactv = np.empty(N, dtype=object)
    for i in range(N):
        exactv[i] = fn(fa[i], fb[i])
    ok, idx = _bound_ok(r, exactv, K)
    assert ok, f"entry {idx} outside 2^-{51 * K}"


@pytest.mark.parametrize("K", KS)
@pytest.mark.parametrize("C", [1, 2])
def test_md_div(K, C):
    N = 24
    a = wl.random_md((N,), K, C, 77 + K)
    b = wl.random_md((N,), K, C, 78 + K)
    b[0, 0, :4] = 2.0 ** np.arange(-3, 1)  # exact powers of two
    r = oracle.md_binary("div", a, b)
    fa, fb = ex.arr_to_fr(a), ex.arr_to_fr(b)
    exactv = np.empty(N, dtype=object)
    for i in range(N):
        exactv[i] = ex.div(fa[i], fb[i])
    ok, idx = _bound_ok(r, exactv, K, slack=4)
    assert ok, f"entry {idx}"


def test_md_div_by_zero_is_reported():
    a = np.ones((2, 1, 1))
    b = np.zeros((2, 1, 1))
    with pytest.raises(oracle.OracleError):
        oracle.md_binary("div", a, b)


@pytest.mark.parametrize("K", KS)
def test_md_sqrt(K):
    N = 24
    a = np.abs(wl.random_md((N,), K, 1, 91 + K))[:, 0]
    a[:, 0] = 0.0
    a[0, 1] = 4.0
    a[1:, 1] = 0.0          # sqrt(4) = 2 exactly
    a[0, 2] = 2.0
    a[1:, 2] = 0.0          # sqrt(2): irrational, checked via r^2
    a[0, 3] *= 2.0 ** 200
    r = oracle.md_sqrt(a)
    assert np.all(r[:, 0] == 0.0)
    assert r[0, 1] == 2.0 and np.all(r[1:, 1] == 0.0)
    bound = Fr(4) * Fr(2) ** (-51 * K)
    for i in range(1, N):
        av = ex.md_to_fr(a[:, i])
        rv = ex.md_to_fr(r[:, i])
        assert rv > 0
        # |r - sqrt a| = |r^2 - a| / (r + sqrt a) ~ |r^2 - a| / (2 r)
        assert abs(rv * rv - av) <= 2 * bound * av, i


@pytest.mark.parametrize("K", KS)
def test_md_outputs_are_nonoverlapping(K):
    a, b = _random_pair(K, 1, 40, 5 + K)
    for op in ("add", "mul", "div"):
        if op == "div":
            b = np.where(b == 0.0, 1.0, b)
        r = oracle.md_binary(op, a, b)[:, 0]
        for l in range(K - 1):
            lead = np.abs(r[l])
            nxt = np.abs(r[l + 1])
            ok = (nxt <= 2.0 * np.spacing(lead)) | (lead == 0.0) & (nxt == 0.0)
            assert np.all(ok), (op, l)
