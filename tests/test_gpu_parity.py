"""GPU path (through the C-ABI) against the CPU oracle, element by element,
on seeded inputs: evaluation and differentiation, the block Toeplitz solve
and whole Newton runs, over limbs, real/complex data, ragged degrees and
sizes that span several warps and waves, and the degenerate cases.

Tolerances: the stated per-coefficient bars 1e-28 (dd), 1e-58 (qd) and
1e-118 (od), normalised by max(|y_k|, series or matrix scale)."""
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


def _newton(md, s):
    return md.Newton(s)


EVAL_CASES = [
    # K, C, n, d, monomials per equation, kmin, kmax
    (1, 1, 5, 7, 3, 1, 3),
    (2, 1, 8, 15, 4, 3, 3),
    (2, 1, 3, 0, 2, 1, 3),       # d = 0: one coefficient (plain md products)
    (2, 2, 6, 10, 3, 1, 4),      # odd D = 11: ragged lane groups
    (4, 1, 17, 31, 5, 2, 8),     # n not a multiple of the warp
    (4, 2, 5, 20, 3, 1, 5),
    (8, 1, 4, 63, 2, 1, 5),      # D = 64: one product per warp
    (8, 2, 3, 12, 2, 2, 4),
]


@pytest.mark.parametrize("K,C,n,d,mpe,kmin,kmax", EVAL_CASES)
def test_evaluate_matches_oracle(md, K, C, n, d, mpe, kmin, kmax):
    cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=mpe, kmin=kmin, kmax=kmax, index=700 + K + 10 * C + n)
    s, xstar, x0 = planted(cfg)
    x = wl.random_md((n, d + 1), K, C, 31 + n, unit_circle=(C == 2))
    f_ref, A_ref = oracle.evaluate(s, x)
    nw = _newton(md, s)
    f, A = nw.evaluate(x)
    assert mt.matrix_rel_error(to_np(f), f_ref) <= TOL[K]
    assert mt.matrix_rel_error(to_np(A), A_ref) <= TOL[K]


def test_evaluate_powers_and_single_variable_monomials(md):
    """Repeated variables are powers (their partials add up); one-variable
    monomials have the coefficient series as partial."""
    K, C, n, d = 4, 1, 3, 9
    D = d + 1
    eq = np.array([0, 0, 1, 2, 2], np.int32)
    vptr = np.array([0, 3, 4, 6, 7, 9], np.int32)
    vidx = np.array([0, 0, 1, 2, 1, 1, 2, 0, 2], np.int32)   # x0^2 x1, x2, x1^2, x2, x0 x2
    coeff = wl.random_md((5, D), K, C, 5)
    s = wl.System(K, C, n, d, eq, vptr, vidx, coeff, wl.random_md((n, D), K, C, 6))
    x = wl.random_md((n, D), K, C, 7)
    f_ref, A_ref = oracle.evaluate(s, x)
    f, A = _newton(md, s).evaluate(x)
    assert mt.matrix_rel_error(to_np(f), f_ref) <= TOL[K]
    assert mt.matrix_rel_error(to_np(A), A_ref) <= TOL[K]


def test_speelpenning_on_gpu(md):
    """prod_{i<8} x_i at x_i = 1 + t: binomial coefficients, exactly."""
    from math import comb
    K, k, D = 4, 8, 12
    s = wl.System(K, 1, k, D - 1, np.zeros(1, np.int32), np.array([0, k], np.int32), np.arange(k, dtype=np.int32),
                  np.zeros((K, 1, 1, D)), np.zeros((K, 1, k, D)))
    s.coeff[0, 0, 0, 0] = 1.0
    x = np.zeros((K, 1, k, D))
    x[0, 0, :, 0] = 1.0
    x[0, 0, :, 1] = 1.0
    f, A = _newton(md, s).evaluate(x)
    f, A = to_np(f), to_np(A)
    for j in range(D):
        assert f[0, 0, 0, j] == comb(k, j) and np.all(f[1:, 0, 0, j] == 0)
        assert np.all(A[0, 0, j, 0, :] == comb(k - 1, j)) and np.all(A[1:, 0, j, 0, :] == 0)


SOLVE_CASES = [(2, 1, 7, 15), (4, 1, 33, 31), (4, 2, 9, 7), (8, 1, 5, 20), (8, 2, 4, 5), (2, 1, 1, 0)]


@pytest.mark.parametrize("K,C,n,d", SOLVE_CASES)
def test_solve_matches_oracle(md, K, C, n, d):
    D = d + 1
    A = wl.random_md((D, n, n), K, C, 40 + n, unit_circle=False)
    for i in range(n):
        A[0, 0, 0, i, i] += n
    b = wl.random_md((n, D), K, C, 41 + n)
    dx_ref = oracle.solve(A, b)
    # any system gives a context of the right shape
    cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=1, kmin=1, kmax=1, index=800)
    s, _, _ = planted(cfg, with_cst=False)
    dx = _newton(md, s).solve(A, b)
    assert np.max(mt.series_rel_error(to_np(dx), dx_ref)) <= TOL[K]


@pytest.mark.parametrize("K,C", [(2, 1), (4, 1), (8, 1), (2, 2), (4, 2), (8, 2)])
def test_series_division_n1(md, K, C):
    """n = 1: the block Toeplitz solve is the series quotient b(t) / a(t);
    it exercises the 1x1 reflector, 1/R and the reciprocal and square root
    kernels at full precision over 64 coefficients."""
    D = 64
    A = wl.random_md((D, 1, 1), K, C, 900 + K + C, unit_circle=(C == 2))
    A[0, 0, 0] += 2.0 if C == 1 else 0.0
    A[:, :, 1:] *= (0.25 ** np.arange(1, D))[:, None, None]  # no zero of a(t) near the unit disk
    b = wl.random_md((1, D), K, C, 901 + K)
    dx_ref = oracle.solve(A, b)
    cfg = wl.small_config(K, C, n=1, d=D - 1, mono_per_eq=1, kmin=1, kmax=1, index=806)
    s, _, _ = planted(cfg, with_cst=False)
    dx = _newton(md, s).solve(A, b)
    assert np.max(mt.series_rel_error(to_np(dx), dx_ref)) <= TOL[K]


def test_singular_A0_is_reported(md):
    K, C, n, d = 2, 1, 4, 3
    A = wl.random_md((d + 1, n, n), K, C, 3)
    A[:, :, 0, :, 2] = 0.0        # zero column of A0
    b = wl.random_md((n, d + 1), K, C, 4)
    cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=1, kmin=1, kmax=1, index=801)
    s, _, _ = planted(cfg, with_cst=False)
    nw = _newton(md, s)
    with pytest.raises(md.MdnError) as e:
        nw.solve(A, b)
    assert e.value.status == md.MDN_ESINGULAR


def test_nonfinite_series_is_reported(md):
    cfg = wl.small_config(2, 1, n=4, d=5, index=802)
    s, xstar, x0 = planted(cfg)
    nw = _newton(md, s)
    x0 = x0.copy()
    x0[0, 0, 1, 0] = np.nan
    nw.set_series(x0)
    with pytest.raises(md.MdnError) as e:
        nw.newton(1)
    assert e.value.status == md.MDN_ENONFINITE


NEWTON_CASES = [
    wl.small_config(2, 1, n=4, d=7, mono_per_eq=3, kmin=1, kmax=3, steps=6, index=500),
    wl.small_config(4, 1, n=5, d=9, mono_per_eq=3, kmin=2, kmax=4, steps=7, index=501),
    wl.small_config(8, 2, n=3, d=5, mono_per_eq=2, kmin=1, kmax=3, steps=8, index=502),
    wl.small_config(4, 2, n=6, d=13, mono_per_eq=3, kmin=1, kmax=4, steps=7, index=503),
    wl.small_config(2, 1, n=40, d=15, mono_per_eq=4, kmin=2, kmax=6, steps=6, index=504),
]


@pytest.mark.parametrize("cfg", NEWTON_CASES, ids=lambda c: c.name)
def test_newton_matches_oracle_and_plant(md, cfg):
    s, xstar, x0 = planted(cfg)
    x_ref, h_ref = oracle.newton(s, x0, cfg.steps)
    nw = _newton(md, s)
    nw.set_series(x0)
    hist = nw.newton(cfg.steps)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, x_ref)) <= cfg.tol
    assert np.max(mt.series_rel_error(x, xstar)) <= cfg.tol
    _check_history(hist, h_ref, cfg.K, s.n * s.D, cfg.tol)


def _check_history(hist, h_ref, K, entries, tol):
    """The three history columns against the oracle's (Section 2 pseudo
    code): ||f||_1 and ||dx||_1 where they are above the rounding level of
    the series (there the two sides agree to far more than 1e-10), the
    monitor ||b - A dx||_1 at the md rounding level of the step on both
    sides (the residual of a computed solve is rounding noise, so its value
    is not reproducible across implementations, only its size)."""
    assert hist.shape == h_ref.shape
    big0 = h_ref[:, 0] > 1e-6
    assert np.allclose(hist[big0, 0], h_ref[big0, 0], rtol=1e-10)
    big2 = h_ref[:, 2] > tol ** 0.5
    assert big2[0]
    assert np.allclose(hist[big2, 2], h_ref[big2, 2], rtol=1e-10)
    eps = 2.0 ** (12 - 52 * K)
    bound = eps * entries * np.maximum(1.0, h_ref[:, 0])
    assert np.all(hist[:, 1] <= bound) and np.all(h_ref[:, 1] <= bound)
    assert hist[-1, 0] < 1e3 * tol


@pytest.mark.parametrize("K", [2, 4])
def test_newton_sqrt_one_plus_t(md, K):
    s, sol, x0 = ts.sqrt_system(K, 15 if K == 2 else 31)
    nw = _newton(md, s)
    nw.set_series(x0)
    nw.newton(6 if K == 2 else 7)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, ts.solution_md(sol, K, 1))) <= TOL[K]


def test_newton_two_column_complex(md):
    from fractions import Fraction as Fr
    alphas = [(Fr(3, 5), Fr(4, 5)), (Fr(-4, 5), Fr(3, 5)), (Fr(-1), Fr(0))]
    c1 = [(Fr(3, 4), Fr(1, 4)), (Fr(-5, 4), Fr(0)), (Fr(1, 2), Fr(-1, 2))]
    c2 = [(Fr(3, 8), Fr(0)), (Fr(1), Fr(1, 8)), (Fr(-5, 8), Fr(1, 4))]
    s, sol, x0 = ts.two_column_system(4, 2, alphas, c1, c2, 31)
    nw = _newton(md, s)
    nw.set_series(x0)
    nw.newton(8)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, ts.solution_md(sol, 4, 2))) <= TOL[4]


@pytest.mark.parametrize("K,C", [(8, 2), (8, 1), (4, 1), (2, 1)])
def test_solve_late_updates_matches_oracle(md, K, C):
    """Stated-accuracy variant: stages k >= 10 form their updates in K/2
    limbs.  Early stages meet the K-limb tolerance against the oracle's
    variant; late stages agree to the K/2-limb rounding level (the two sides
    round the K/2-limb sums differently) and really differ from the plain
    solve at that level."""
    n, d, late = 9, 20, 10
    A = wl.random_md((d + 1, n, n), K, C, 60 + K, unit_circle=False)
    for i in range(n):
        A[0, 0, 0, i, i] += n
    b = wl.random_md((n, d + 1), K, C, 61 + K)
    ref = oracle.solve(A, b, late=(late, K // 2))
    cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=1, kmin=1, kmax=1, index=807)
    s, _, _ = planted(cfg, with_cst=False)
    nw = _newton(md, s)
    nw.set_late_updates(late, K // 2)
    dx = to_np(nw.solve(A, b))
    eps_half = 2.0 ** (-52 * (K // 2))
    e = mt.series_rel_error(dx, ref)
    assert e[:, :late].max() <= TOL[K]
    assert e[:, late:].max() <= 1e4 * eps_half
    assert mt.series_rel_error(dx, oracle.solve(A, b))[:, late:].max() >= 1e-6 * eps_half
    # switched off again: the plain solve
    nw.set_late_updates(1, K)
    assert np.max(mt.series_rel_error(to_np(nw.solve(A, b)), oracle.solve(A, b))) <= TOL[K]


def test_set_late_updates_rejects_bad_arguments(md):
    cfg = wl.small_config(4, 1, n=3, d=5, mono_per_eq=1, kmin=1, kmax=1, index=808)
    s, _, _ = planted(cfg, with_cst=False)
    nw = _newton(md, s)
    for first, limbs in [(0, 2), (3, 3), (3, 1), (3, 8)]:
        with pytest.raises(md.MdnError) as e:
            nw.set_late_updates(first, limbs)
        assert e.value.status == md.MDN_EINVAL


def test_newton_late_updates_recovers_plant(md):
    cfg = wl.small_config(8, 2, n=6, d=15, mono_per_eq=3, kmin=1, kmax=4, steps=9, index=506)
    s, xstar, x0 = planted(cfg)
    x_ref, _ = oracle.newton(s, x0, cfg.steps, late=(8, 4))
    nw = _newton(md, s)
    nw.set_late_updates(8, 4)
    nw.set_series(x0)
    nw.newton(cfg.steps)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, xstar)) <= cfg.tol
    assert np.max(mt.series_rel_error(x, x_ref)) <= cfg.tol


RESIDUAL_CASES = [(1, 1, 6, 9), (2, 1, 7, 15), (4, 1, 33, 31), (4, 2, 9, 7), (8, 1, 5, 20), (8, 2, 4, 5),
                  (2, 1, 1, 0)]


@pytest.mark.parametrize("K,C,n,d", RESIDUAL_CASES)
def test_residual_matches_oracle(md, K, C, n, d):
    """mdn_residual (r_k = b_k - sum_{j<=k} A_j dx_{k-j}, Sections 5.4 and 6)
    against the oracle's exact-then-round residual, entry by entry, for a dx
    perturbed off the solution so that r sits far above the rounding level
    (2^(-26K) of the terms, against a tolerance of 2^(8-53K) of them); its
    norm and the sampled norm over a subset of rows (scaled by n / rows)."""
    D = d + 1
    A = wl.random_md((D, n, n), K, C, 70 + n + K)
    for i in range(n):
        A[0, 0, 0, i, i] += n
    b = wl.random_md((n, D), K, C, 71 + n)
    dx = oracle.solve(A, b)
    pert = wl.random_md((n, D), K, C, 72 + n) * 2.0 ** (-26 * K)
    dx = oracle.md_binary("add", dx.reshape(K, C, -1), pert.reshape(K, C, -1)).reshape(dx.shape)
    r_ref, norm_ref = oracle.toeplitz_residual(A, b, dx)
    cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=1, kmin=1, kmax=1, index=809)
    s, _, _ = planted(cfg, with_cst=False)
    nw = _newton(md, s)
    r, norm = nw.residual(A, b, dx)
    r = to_np(r)
    # size of the terms of each entry (leading doubles)
    Am = mt.magnitude(A[0])  # [D, n, n]
    xm = mt.magnitude(dx[0])  # [n, D]
    size = mt.magnitude(b[0]).copy()
    for k in range(D):
        for j in range(k + 1):
            size[:, k] += Am[j] @ xm[:, k - j]
    err = mt.magnitude(mt.md_diff(r, r_ref))
    assert np.all(err <= 2.0 ** (8 - 53 * K) * size)
    assert np.median(mt.magnitude(mt.md_value(r_ref)) / size) >= 2.0 ** (-26 * K - 8)
    # the norms sum leading doubles: they agree to the entries' error bound
    slack = 2.0 ** (8 - 53 * K) * size
    assert abs(norm - norm_ref) <= 1e-12 * norm_ref + slack.sum()
    rows = [n - 1] if n == 1 else [0, n - 1]
    nw.set_residual_rows(rows)
    _, part = nw.residual(A, b, dx, want_r=False)
    _, part_ref = oracle.toeplitz_residual(A, b, dx, rows=rows)
    assert abs(part - part_ref) <= 1e-12 * part_ref + n / len(rows) * slack[rows].sum()


def test_sampled_residual_monitor(md):
    """The monitor on a subset of rows is that subset's share scaled by
    n / rows: the full monitor splits exactly into a sample and its
    complement; the iterates and the other norms do not depend on it."""
    n = 12
    cfg = wl.small_config(4, 1, n=n, d=9, mono_per_eq=3, kmin=1, kmax=4, steps=3, index=509)
    s, xstar, x0 = planted(cfg)
    nw = _newton(md, s)

    def run(rows):
        nw.set_residual_rows(rows)
        nw.set_series(x0)
        return nw.newton(3)

    full = run([])
    assert np.array_equal(run(list(range(n))), full)
    rest = [i for i in range(n) if i != 5]
    h_rest, h_one = run(rest), run([5])
    np.testing.assert_allclose((n - 1) / n * h_rest[:, 1] + h_one[:, 1] / n, full[:, 1], rtol=1e-12)
    assert np.array_equal(h_one[:, [0, 2]], full[:, [0, 2]])
    assert np.all(h_one[:, 1] > 0)
    with pytest.raises(md.MdnError):
        nw.set_residual_rows([1, 1])
    with pytest.raises(md.MdnError):
        nw.set_residual_rows([n])


@pytest.mark.parametrize("K,C,n,d,first,steps", [(2, 1, 5, 15, 4, 12), (4, 1, 9, 31, 5, 14),
                                                 (8, 2, 4, 15, 6, 14), (4, 1, 3, 7, 2, 3)])
def test_staggered_newton_matches_oracle(md, K, C, n, d, first, steps):
    """Staggered orders with the QR once against the oracle's staggered
    Newton: the same series after every schedule, the plant at the end."""
    cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=3, kmin=1, kmax=4, index=560 + K + n)
    s, xstar, x0 = planted(cfg)
    x_ref, h_ref, orders = oracle.newton_staggered(s, x0, steps, first)
    nw = _newton(md, s)
    nw.set_stagger(first)
    nw.set_series(x0)
    hist = nw.newton(steps)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, x_ref)) <= TOL[K]
    big = h_ref[:, 0] > 1e-6
    assert np.allclose(hist[big, 0], h_ref[big, 0], rtol=1e-10)
    if orders[-1] == d + 1 and steps >= 12:
        assert np.max(mt.series_rel_error(x, xstar)) <= TOL[K]
    else:  # coefficients beyond the last order are untouched
        assert np.array_equal(x[..., orders[-1]:], x0[..., orders[-1]:])
    # back to the plain method
    nw.set_stagger(0)
    nw.set_series(x0)
    nw.newton(2)
    x2_ref, _ = oracle.newton(s, x0, 2)
    assert np.max(mt.series_rel_error(to_np(nw.series()), x2_ref)) <= TOL[K]


def test_evaluation_only_context_beyond_the_qr_limit(md):
    """n = 1100 > MDN_MAX_N: the paper's one-column system (monomial i =
    x_0...x_i, up to 1100 variables) evaluates, rows of f and of the
    Jacobian match the oracle; the solve calls refuse.  Quad double: a
    product of 60 series of mixed-sign exponentials cancels by ~1e4, which a
    double double result shows at its last digits (2e-28 against 1e-28)."""
    K, n, d = 4, 1100, 11
    s, x = wl.one_column_system(n, d, K)
    nw = _newton(md, s)
    f, A = nw.evaluate(x)
    f, A = to_np(f), to_np(A)
    rows = [0, 7, 60]
    keep = np.isin(s.eq, rows)
    sub = wl.System(s.K, s.C, s.n, s.d, s.eq[keep], None, None, s.coeff[:, :, keep], s.cst)
    sizes = np.diff(s.vptr)[keep]
    sub.vptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    sub.vidx = np.concatenate([s.vidx[s.vptr[m]:s.vptr[m + 1]] for m in np.nonzero(keep)[0]]).astype(np.int32)
    f_ref, A_ref = oracle.evaluate(sub, x)
    assert mt.matrix_rel_error(f[:, :, rows], f_ref[:, :, rows]) <= TOL[K]
    assert mt.matrix_rel_error(A[:, :, :, rows], A_ref[:, :, :, rows]) <= TOL[K]
    nw.set_series(x)
    with pytest.raises(md.MdnError) as e:
        nw.newton(1)
    assert e.value.status == md.MDN_EINVAL


def test_newton_at_the_largest_n(md):
    """n = MDN_MAX_N_DATAFLOW = 192 (the dataflow QR launch at its largest:
    120 blocks, one per SM): Newton against the oracle and the plant; one
    past the evaluation limit is refused at creation."""
    cfg = wl.small_config(2, 1, n=192, d=3, mono_per_eq=1, kmin=1, kmax=2, steps=5, index=512)
    s, xstar, x0 = planted(cfg)
    x_ref, _ = oracle.newton(s, x0, cfg.steps)
    nw = _newton(md, s)
    nw.set_series(x0)
    nw.newton(cfg.steps)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, x_ref)) <= cfg.tol
    assert np.max(mt.series_rel_error(x, xstar)) <= cfg.tol
    with pytest.raises(md.MdnError) as e:
        md.mdn_create(2, 0, 4097, 3)
    assert e.value.status == md.MDN_EINVAL
