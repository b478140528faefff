"""Pins of the oracle's adjoint (gradients of a loss of the converged series
with respect to the coefficient series) and of the Fabry-ratio loss.

The loss is checked against exact rationals.  The adjoint gradient of a
double double system is checked against central differences of the loss in
octo double: the system is promoted exactly to 8 limbs, one coefficient (or
all of them along a random direction) is moved by +-h, h = 1e-20, Newton is
rerun in octo double, and (L+ - L-) / 2h is formed exactly.  The truncation
error of the quotient is O(h^2), far below the double double gradient's
own rounding."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import exact as ex

H = Fr(1e-20)


def _converged_dd(index, n=3, d=5):
    cfg = wl.small_config(2, 1, n=n, d=d, mono_per_eq=2, kmin=1, kmax=3, steps=8, index=index)
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    x, _ = oracle.newton(s, x0, 8)
    return s, x


def _promote(a, K=8):
    out = np.zeros((K,) + a.shape[1:])
    out[:a.shape[0]] = a
    return out


def _loss_od(s, x_start, coeff8):
    s8 = wl.System(8, 1, s.n, s.d, s.eq, s.vptr, s.vidx, coeff8, _promote(s.cst))
    x8, _ = oracle.newton(s8, _promote(x_start), 5)
    L, _ = oracle.fabry_loss(x8)
    return ex.md_to_fr(L)


def _shift(coeff8, m, j, delta: Fr):
    v = ex.md_to_fr(coeff8[:, 0, m, j]) + delta
    coeff8[:, 0, m, j] = ex.fr_to_md(v, 8)


def test_fabry_loss_exact():
    s, x = _converged_dd(520)
    L, g = oracle.fabry_loss(x)
    d = s.d
    X = ex.arr_to_fr(x)
    exact = sum((X[i, d] * X[i, d] for i in range(s.n)), Fr(0)) + X[0, d - 1] / X[0, d]
    assert abs(ex.md_to_fr(L) - exact) <= abs(exact) * Fr(2) ** -100
    G = ex.arr_to_fr(g)
    for i in range(s.n):
        for k in range(d + 1):
            want = Fr(0)
            if k == d:
                want = 2 * X[i, d] - (X[0, d - 1] / (X[0, d] * X[0, d]) if i == 0 else 0)
            if k == d - 1 and i == 0:
                want = 1 / X[0, d]
            assert abs(G[i, k] - want) <= abs(want) * Fr(2) ** -100


@pytest.mark.parametrize("index", [521, 522])
def test_adjoint_against_octo_double_central_differences(index):
    s, x = _converged_dd(index)
    _, g = oracle.fabry_loss(x)
    grad = oracle.adjoint(s, x, g)
    scale = float(np.max(np.abs(grad[0, 0])))
    coeff8 = _promote(s.coeff)
    rng = np.random.default_rng(index)
    picks = [(int(rng.integers(s.M)), int(rng.integers(s.D))) for _ in range(6)]
    for m, j in picks:
        cp, cm = coeff8.copy(), coeff8.copy()
        _shift(cp, m, j, H)
        _shift(cm, m, j, -H)
        fd = (_loss_od(s, x, cp) - _loss_od(s, x, cm)) / (2 * H)
        adj = ex.md_to_fr(grad[:, 0, m, j])
        assert abs(fd - adj) <= Fr(1e-24) * max(abs(adj), Fr(1e-6) * Fr(scale)), (m, j, float(fd), float(adj))
    # a random direction through every coefficient
    u = rng.choice([-1, 1], size=(s.M, s.D))
    cp, cm = coeff8.copy(), coeff8.copy()
    for m in range(s.M):
        for j in range(s.D):
            _shift(cp, m, j, H * int(u[m, j]))
            _shift(cm, m, j, -H * int(u[m, j]))
    fd = (_loss_od(s, x, cp) - _loss_od(s, x, cm)) / (2 * H)
    adj = sum((ex.md_to_fr(grad[:, 0, m, j]) * int(u[m, j]) for m in range(s.M) for j in range(s.D)), Fr(0))
    assert abs(fd - adj) <= Fr(1e-24) * abs(adj)


def test_adjoint_of_a_linear_system_is_exact_rational():
    """All monomials of one variable: f = C x + cst with coefficient series,
    so lambda solves the transposed block Toeplitz system exactly; compare
    with an exact rational solve on a tiny case."""
    K, n, d = 2, 2, 3
    D = d + 1
    eq = np.array([0, 0, 1, 1], np.int32)
    vptr = np.array([0, 1, 2, 3, 4], np.int32)
    vidx = np.array([0, 1, 0, 1], np.int32)
    coeff = wl.random_md((4, D), K, 1, 12)
    coeff[0, 0, 0, 0] += 4.0
    coeff[0, 0, 3, 0] += 4.0
    s = wl.System(K, 1, n, d, eq, vptr, vidx, coeff, None)
    x = wl.random_md((n, D), K, 1, 13)
    g = wl.random_md((n, D), K, 1, 14)
    grad = oracle.adjoint(s, x, g)
    # exact: A_j[i][v] = coefficient j of the monomial of equation i in x_v
    Cf = ex.arr_to_fr(coeff)
    A = [[[Cf[2 * i + v, j] for v in range(n)] for i in range(n)] for j in range(D)]
    G = ex.arr_to_fr(g)
    lam = [[Fr(0)] * D for _ in range(n)]
    for k in range(d, -1, -1):
        r = [G[i, k] - sum((A[j][l][i] * lam[l][k + j] for j in range(1, d - k + 1) for l in range(n)), Fr(0))
             for i in range(n)]
        # A_0^T lam_k = r (2x2, exact)
        a, b, c, e = A[0][0][0], A[0][1][0], A[0][0][1], A[0][1][1]  # A0^T = [[a, b], [c, e]]
        det = a * e - b * c
        lam[0][k] = (e * r[0] - b * r[1]) / det
        lam[1][k] = (a * r[1] - c * r[0]) / det
    X = ex.arr_to_fr(x)
    for m in range(4):
        i, v = int(eq[m]), int(vidx[m])
        for j in range(D):
            want = -sum((lam[i][k] * X[v, k - j] for k in range(j, D)), Fr(0))
            got = ex.md_to_fr(grad[:, 0, m, j])
            assert abs(got - want) <= max(abs(want), Fr(1)) * Fr(2) ** -98
