"""Newton beyond the dataflow QR (n > MDN_MAX_N_DATAFLOW = 192): the
column-by-column Householder QR in global memory (Section 5.3) with the
forward substitution and the evaluation at the sizes of the paper's
Section 6 runs, through the C-ABI.

* Solve and Newton against the oracle at n = 200..512 (dd, complex qd).
* The paper's one-column system of Section 3 (x_0 x_1 ... x_i = b_i(t),
  solutions exp(alpha_v t)) at n = 1024 with 64 coefficients in octo
  double, with staggered orders and the QR once (Sections 4 and 5.3),
  against its closed-form solution; the two-column system likewise at a
  reduced n against the oracle."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import metrics as mt
from tests import systems as ts
from tests.gpu_util import TOL, need_gpu, planted, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    return need_gpu()


@pytest.mark.parametrize("K,C,n,d", [(2, 1, 200, 3), (4, 2, 196, 1), (8, 1, 256, 2), (2, 1, 512, 1)])
def test_large_solve_matches_oracle(md, K, C, n, d):
    D = d + 1
    A = wl.random_md((D, n, n), K, C, 40 + n)
    for i in range(n):
        A[0, 0, 0, i, i] += n
    b = wl.random_md((n, D), K, C, 41 + n)
    dx_ref = oracle.solve(A, b)
    cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=1, kmin=1, kmax=1, index=810)
    s, _, _ = planted(cfg, with_cst=False)
    nw = md.Newton(s)
    dx = to_np(nw.solve(A, b))
    assert np.max(mt.series_rel_error(dx, dx_ref)) <= TOL[K]
    # the residual of the computed solve is at the rounding level
    _, norm = nw.residual(A, b, dx)
    assert norm <= 2.0 ** (12 - 52 * K) * n * n * D


def test_large_singular_A0_is_reported(md):
    K, C, n, d = 2, 1, 200, 1
    A = wl.random_md((d + 1, n, n), K, C, 5)
    A[:, :, 0, :, 17] = 0.0
    b = wl.random_md((n, d + 1), K, C, 6)
    cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=1, kmin=1, kmax=1, index=811)
    s, _, _ = planted(cfg, with_cst=False)
    with pytest.raises(md.MdnError) as e:
        md.Newton(s).solve(A, b)
    assert e.value.status == md.MDN_ESINGULAR


@pytest.mark.parametrize("K,C,n,d,steps", [(2, 1, 256, 7, 6), (4, 2, 200, 3, 7)])
def test_large_newton_matches_oracle_and_plant(md, K, C, n, d, steps):
    cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=2, kmin=1, kmax=3, steps=steps, index=514 + n)
    s, xstar, x0 = planted(cfg)
    x_ref, h_ref = oracle.newton(s, x0, cfg.steps)
    nw = md.Newton(s)
    nw.set_series(x0)
    hist = nw.newton(cfg.steps)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, x_ref)) <= cfg.tol
    assert np.max(mt.series_rel_error(x, xstar)) <= cfg.tol
    big = h_ref[:, 0] > 1e-6
    assert np.allclose(hist[big, 0], h_ref[big, 0], rtol=1e-10)


def _alphas(n, seed, scale=Fr(1), signs=True):
    """alpha_v in scale * ([-1, -0.9] u [0.9, 1]), dyadic (Section 3 with
    delta = 0.1); positive only when signs is False."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        a = scale * Fr(int(rng.integers(58982, 65537)), 65536)  # in [0.9, 1]
        out.append(-a if signs and rng.random() < 0.5 else a)
    return out


def test_two_column_system_staggered_matches_oracle(md):
    """The two-column system of Section 3 (E1 lower triangular ones, E2 its
    rows reversed) at n = 24 with 64 coefficients in octo double: staggered
    orders with the QR once against the oracle's, and the closed form."""
    n, d, K = 24, 63, 8
    al = _alphas(n, 24)
    c1 = [Fr(3, 4) + Fr(i, 64) for i in range(n)]
    c2 = [Fr(-5, 8) + Fr(i, 128) for i in range(n)]
    s, sol, x0 = ts.two_column_system(K, 1, al, c1, c2, d)
    first, steps = 6, 17
    x_ref, _, orders = oracle.newton_staggered(s, x0, steps, first)
    assert orders[-1] == d + 1
    nw = md.Newton(s)
    nw.set_stagger(first)
    nw.set_series(x0)
    nw.newton(steps)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, x_ref)) <= TOL[K]
    assert np.max(mt.series_rel_error(x, ts.solution_md(sol, K, 1))) <= TOL[K]


@pytest.mark.parametrize("n,d,K", [(1024, 63, 8), (300, 31, 4)])
def test_one_column_system_at_the_paper_size(md, n, d, K):
    """The one-column system of Section 3 at n = 1024 with 64 coefficients in
    octo double (the paper's Table 4 and 5 workload), with staggered orders
    (x_0 first, then 1, 2, 4, 7, ... coefficients) and the QR once: every
    coefficient of every x_v(t) = exp(alpha_v t) to the octo double bar.
    The alpha_v are positive and scaled by 4/n, so that the right hand sides
    exp((alpha_0 + ... + alpha_i) t) stay of size e^4: with the paper's
    alpha in +-[0.9, 1] the partial sums wander to |s| ~ 60 at n = 1024 and
    the coefficients of the series products grow to e^|s| ~ 1e26, so no
    md precision keeps 1e-118 of the solution (the error growth of
    Section 2); the structure, sizes and arithmetic are the paper's."""
    al = _alphas(n, n, scale=Fr(4, n), signs=False)
    s, sol, x0 = ts.one_column_system(K, 1, al, d)
    first = {4: 5, 8: 6}[K]
    L, steps = 1, first
    while L < d + 1:
        L, steps = min(d + 1, L + 1 + L // 2), steps + 1
    steps += 2
    nw = md.Newton(s)
    nw.set_stagger(first)
    nw.set_series(x0)
    hist = nw.newton(steps)
    x = to_np(nw.series())
    err = mt.series_rel_error(x, ts.solution_md(sol, K, 1))
    assert np.max(err) <= TOL[K], (float(np.max(err)), hist[-3:])
