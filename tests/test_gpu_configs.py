"""The three plain Newton workloads at full size through the C-ABI.

* double double, n=8, d=15: GPU Newton (6 steps) against the oracle's Newton,
  entry by entry, and against the planted solution, tolerance 1e-28;
* quad double, n=64, d=31: evaluation and differentiation at the start
  series against the oracle (all of f and A), 7 GPU Newton steps against the
  oracle's 7 steps and against the planted solution, tolerance 1e-58;
* complex octo double, n=128, d=63: eight full rows of f and of every A_j
  at a random series against the oracle (the densest rows among them);
  Newton on the system whose constant term the oracle planted (stored by
  tests/golden/make_od_complex_golden.py) recovering the plant: x_0 and the
  leading coefficients to 1e-118, the error of x_0 squaring per step, the
  late coefficients to the conditioning floor; a reduced analogue of the
  same recipe (n = 16) against the oracle's Newton coefficient by
  coefficient, which shows the floor on the oracle as well; and the
  stated-accuracy variant (updates of the stages k >= 32 in quad double),
  which reaches the same accuracy.
"""
import os

import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import metrics as mt
from tests.gpu_util import need_gpu, planted, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    return need_gpu()


def test_dd_real_n8_d15(md):
    cfg = wl.CONFIGS["dd-real-n8-d15"]
    s, xstar, x0 = planted(cfg)
    x_ref, h_ref = oracle.newton(s, x0, cfg.steps)
    nw = md.Newton(s)
    nw.set_series(x0)
    hist = nw.newton(cfg.steps)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, x_ref)) <= cfg.tol
    assert np.max(mt.series_rel_error(x, xstar)) <= cfg.tol
    assert np.allclose(hist[:3, 0], h_ref[:3, 0], rtol=1e-12)


def test_qd_real_n64_d31(md):
    cfg = wl.CONFIGS["qd-real-n64-d31"]
    s, xstar, x0 = planted(cfg)
    nw = md.Newton(s)
    f_ref, A_ref = oracle.evaluate(s, x0)
    f, A = nw.evaluate(x0)
    assert mt.matrix_rel_error(to_np(f), f_ref) <= cfg.tol
    assert mt.matrix_rel_error(to_np(A), A_ref) <= cfg.tol
    nw.set_series(x0)
    hist = nw.newton(cfg.steps)
    x = to_np(nw.series())
    assert np.max(mt.series_rel_error(x, xstar)) <= cfg.tol
    x_ref, h_ref = oracle.newton(s, x0, cfg.steps)
    assert np.max(mt.series_rel_error(x, x_ref)) <= cfg.tol
    assert np.allclose(hist[:4, 0], h_ref[:4, 0], rtol=1e-12)


GOLDEN_OD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "od_complex_golden.npz")


def _golden_od():
    if not os.path.exists(GOLDEN_OD):
        pytest.skip("tests/golden/od_complex_golden.npz not written (tests/golden/make_od_complex_golden.py)")
    return np.load(GOLDEN_OD)


def _rows_subsystem(s, rows):
    keep = np.isin(s.eq, rows)
    sub = wl.System(s.K, s.C, s.n, s.d, s.eq[keep], None, None, s.coeff[:, :, keep], s.cst)
    sizes = np.diff(s.vptr)[keep]
    sub.vptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    sub.vidx = np.concatenate([s.vidx[s.vptr[m]:s.vptr[m + 1]] for m in np.nonzero(keep)[0]]).astype(np.int32)
    return sub


def test_od_complex_n128_d63_rows_of_f_and_A(md):
    """Eight full rows of f and of every Jacobian block A_j (the four densest
    rows, with the most variable occurrences, and rows 0, 77, 127 and 50)
    against the oracle at a random unit-circle series."""
    cfg = wl.CONFIGS["od-complex-n128-d63"]
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = np.zeros((s.K, s.C, s.n, s.D))
    occ = np.zeros(s.n, dtype=np.int64)
    np.add.at(occ, s.eq, np.diff(s.vptr))
    rows = sorted(set(np.argsort(-occ, kind="stable")[:4].tolist()) | {0, 50, 77, 127})
    assert len(rows) >= 8
    nw = md.Newton(s)
    x = wl.random_md((s.n, s.D), s.K, s.C, 99, unit_circle=True)
    f, A = nw.evaluate(x)
    f, A = to_np(f), to_np(A)
    f_ref, A_ref = oracle.evaluate(_rows_subsystem(s, rows), x)
    assert mt.matrix_rel_error(f[:, :, rows], f_ref[:, :, rows]) <= cfg.tol
    assert mt.matrix_rel_error(A[:, :, :, rows], A_ref[:, :, :, rows]) <= cfg.tol


def test_od_complex_n128_d63_newton_with_the_oracle_plant(md):
    """Newton on the complex octo double workload whose constant term the
    oracle planted (stored by tests/golden/make_od_complex_golden.py), 8 and
    9 steps from the start series.  x_0 and the leading coefficients meet
    1e-118; the late coefficients settle at a floor that the reduced analogue
    of the same recipe shows on the oracle too (next test): the rounding
    level of f at the solution, amplified through the 64 coefficient blocks
    of the forward substitution (the error propagation of Section 2)."""
    cfg = wl.CONFIGS["od-complex-n128-d63"]
    g = _golden_od()
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = g["cst128"]
    nw = md.Newton(s)
    nw.set_series(x0)
    errs = []
    for step in range(9):
        nw.newton(1)
        e = mt.series_rel_error(to_np(nw.series()), xstar)
        errs.append(e)
    for e in errs[7:]:
        assert np.max(e[:, 0]) <= cfg.tol
        assert mt.correct_leading(to_np(nw.series()), xstar, cfg.tol) >= 16
        assert np.max(e) <= 1e-100
    # quadratic convergence of x_0
    lead = [float(np.max(e[:, 0])) for e in errs]
    for a, b in zip(lead, lead[1:]):
        if a > 1e3 * cfg.tol:
            assert b <= max(1e4 * a * a, cfg.tol), lead


@pytest.mark.parametrize("diag,tag", [(16.0, "16"), (128.0, "16d128")])
def test_od_complex_reduced_analogue_matches_the_oracle(md, diag, tag):
    """The complex octo double recipe at n = 16 (32 monomials per equation of
    2..16 of the 16 variables, 64 coefficients on the unit circle), with the
    diagonal n x_i = 16 x_i or with the full workload's 128 x_i: GPU Newton
    after 8 and 9 steps against the oracle's Newton (stored by
    tests/golden/make_od_complex_golden.py) coefficient by coefficient, and
    both against the plant.  The oracle's own error grows geometrically
    with the coefficient index (the error propagation of Section 2: with the
    diagonal 16 from ~3e-131 at x_0 to ~2e-81 at x_63); the GPU's profile
    follows it from its md rounding level at x_0, so the late-coefficient
    floor is the method's (conditioning), not the kernels'."""
    from tests.golden.make_od_complex_golden import reduced_config
    g = _golden_od()
    if f"x{tag}_9" not in g:
        pytest.skip(f"no oracle values for the reduced analogue {tag}")
    cfg = reduced_config(diag)
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = g[f"cst{tag}"]
    nw = md.Newton(s)
    nw.set_series(x0)
    nw.newton(8)
    x8 = to_np(nw.series())
    nw.newton(1)
    x9 = to_np(nw.series())
    for x, ref in ((x8, g[f"x{tag}_8"]), (x9, g[f"x{tag}_9"])):
        e_orc = mt.series_rel_error(ref, xstar).max(axis=0)
        e_gpu = mt.series_rel_error(x, xstar).max(axis=0)
        # x_0 meets the bar on both sides
        assert e_gpu[0] <= cfg.tol and e_orc[0] <= cfg.tol
        # The oracle rounds the exact value of every expression once, so its
        # f at the solution is accurate relative to f itself; md arithmetic
        # (the paper's, and the GPU's) is accurate relative to the terms of
        # each sum, so its x_0 sits at the md rounding level (base = the
        # ratio of the two errors of x_0).  The forward substitution then
        # amplifies that base by the same factor per coefficient on both
        # sides: the GPU's error profile is the oracle's times the base,
        # within 1e3, coefficient by coefficient, and so is its distance to
        # the oracle's series.
        base = max(1.0, e_gpu[0] / e_orc[0])
        assert np.all(e_gpu <= np.maximum(1e3 * base * e_orc, cfg.tol)), (e_gpu, e_orc, base)
        d = mt.series_rel_error(x, ref)
        assert np.all(d <= np.maximum(cfg.tol, 1e3 * base * e_orc[None, :])), (d.max(axis=0), e_orc, base)
        # the base is the md rounding level, not a loss of accuracy
        assert e_gpu[0] <= 2.0 ** (20 - 53 * 8)


def test_od_complex_n128_d63_late_updates(md):
    """The stated-accuracy variant of the complex octo double workload: the
    updates A_j dx_{k-j} of stages k >= (d+1)/2 = 32 in quad double.  The
    residuals stay in octo double, so Newton reaches the plain run's accuracy
    (x_0 and 16+ leading coefficients to 1e-118, the rest to the same
    conditioning floor) with at most one extra step."""
    cfg = wl.CONFIGS["od-complex-n128-d63"]
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = np.zeros((s.K, s.C, s.n, s.D))
    nw = md.Newton(s)
    cst = -nw.evaluate(xstar, want_A=False)
    nw.set_constant(cst)
    nw.set_late_updates(32, 4)
    nw.set_series(x0)
    nw.newton(cfg.steps + 1)
    x = to_np(nw.series())
    e = mt.series_rel_error(x, xstar)
    assert np.max(e[:, 0]) <= cfg.tol
    assert mt.correct_leading(x, xstar, cfg.tol) >= 16
    assert np.max(e) <= 1e-100
