"""Batched systems through the C-ABI (mdn_batch_*): one persistent launch runs
Newton's method on many independent systems of mixed size, each to the batch
stop rule.  Every system is compared with the oracle's Newton run for the
number of updates the GPU applied to it, and with its planted solution."""
import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import metrics as mt
from tests.gpu_util import TOL, need_gpu, planted, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    return need_gpu()


def _mixed(K, C, shapes, index0):
    out = []
    for q, (n, d, mpe, kmin, kmax) in enumerate(shapes):
        cfg = wl.small_config(K, C, n=n, d=d, mono_per_eq=mpe, kmin=kmin, kmax=kmax, index=index0 + q)
        out.append(planted(cfg) + (cfg,))
    return out


SHAPES = [(3, 3, 2, 1, 3), (5, 7, 3, 1, 4), (8, 10, 3, 2, 5), (4, 0, 2, 1, 3), (1, 6, 2, 1, 2),
          (6, 15, 4, 1, 6), (2, 31, 2, 1, 2)]


@pytest.mark.parametrize("K,C", [(2, 1), (4, 1), (8, 2)])
def test_batch_solve_matches_oracle(md, K, C):
    items = _mixed(K, C, SHAPES, 600 + 10 * K + C)
    systems = [s for s, _, _, _ in items]
    b = md.Batch(systems)
    x0 = b.pack([x0 for _, _, x0, _ in items])
    tol = TOL[K]
    x, steps, flags = b.solve(x0, 12, tol)
    xs = b.unpack(x)
    for q, (s, xstar, x0h, cfg) in enumerate(items):
        assert flags[q] == md.BATCH_CONVERGED, (q, flags[q], steps[q])
        assert 1 <= steps[q] <= 12
        x_ref, _ = oracle.newton(s, x0h, int(steps[q]))
        assert np.max(mt.series_rel_error(xs[q], x_ref)) <= tol, q
        assert np.max(mt.series_rel_error(xs[q], xstar)) <= tol, q
    b.close()


def test_batch_evaluate_matches_oracle(md):
    items = _mixed(4, 1, SHAPES, 640)
    systems = [s for s, _, _, _ in items]
    b = md.Batch(systems)
    xs = [wl.random_md((s.n, s.D), 4, 1, 70 + q) for q, s in enumerate(systems)]
    f = b.unpack(b.evaluate(b.pack(xs)))
    for q, s in enumerate(systems):
        f_ref = oracle.evaluate(s, xs[q], want_A=False)
        assert mt.matrix_rel_error(f[q], f_ref) <= TOL[4]
    b.close()


def test_batch_replay_and_step_cap(md):
    """The captured graph replays to the same bits; a cap of 2 updates stops
    every system after two updates, unconverged, and its x equals the
    oracle's two-step result; max_steps = 0 only evaluates."""
    items = _mixed(2, 1, SHAPES, 660)
    systems = [s for s, _, _, _ in items]
    b = md.Batch(systems, threads_per_block=128, blocks_per_sm=1)
    assert b.tiles() == (128, 1)
    x0 = b.pack([x0 for _, _, x0, _ in items])
    xa, sa, fa = b.solve(x0, 12, TOL[2])
    xb, sb, fb = b.solve(x0, 12, TOL[2])
    assert np.array_equal(to_np(xa), to_np(xb)) and np.array_equal(sa, sb) and np.array_equal(fa, fb)
    x2, s2, f2 = b.solve(x0, 2, TOL[2])
    # two updates, unless the system met the stop rule before (a linear one
    # is solved by its first update)
    assert np.all(((s2 == 2) & (f2 == 0)) | ((s2 <= 2) & (f2 == md.BATCH_CONVERGED)))
    assert np.sum(s2 == 2) >= len(items) - 1
    for q, (s, _, x0h, _) in enumerate(items):
        x_ref, _ = oracle.newton(s, x0h, int(s2[q]))
        assert np.max(mt.series_rel_error(b.unpack(x2)[q], x_ref)) <= TOL[2]
    x_0, s_0, _ = b.solve(x0, 0, TOL[2])
    assert np.all(s_0 == 0) and np.array_equal(to_np(x_0), to_np(x0))
    b.close()


def test_batch_rejects_bad_input(md):
    items = _mixed(2, 1, SHAPES[:2], 680)
    systems = [s for s, _, _, _ in items]
    with pytest.raises(md.MdnError):
        md.Batch(systems, threads_per_block=100)
    bad = systems[1]
    bad.vidx = bad.vidx.copy()
    bad.vidx[0] = bad.n  # out of range
    with pytest.raises(md.MdnError) as e:
        md.Batch(systems)
    assert e.value.status == md.MDN_EINVAL


def test_batch_qd_4096(md):
    """The batched quad double workload at full size: 4096 systems with n in
    {8, 16, 32, 64} and d in {7, 15, 31}, constants planted by the library's
    own evaluation; every system meets the stop rule and recovers its plant
    to 1e-58; three systems (two of the smallest size, one of the largest)
    against the oracle's Newton run of the same number of updates."""
    cfg = wl.BATCH_CONFIGS["qd-real-batch4096"]
    items = wl.batch_planted_systems(cfg)
    systems = [s for s, _, _ in items]
    b = md.Batch(systems)
    xstar = b.pack([xs for _, xs, _ in items])
    b.set_constant(-b.evaluate(xstar))
    x0 = b.pack([x0 for _, _, x0 in items])
    x, steps, flags = b.solve(x0, cfg.max_steps, cfg.tol)
    assert np.all(flags == md.BATCH_CONVERGED), np.unique(flags, return_counts=True)
    xs = b.unpack(x)
    worst = max(float(np.max(mt.series_rel_error(xs[q], items[q][1]))) for q in range(len(items)))
    assert worst <= cfg.tol, worst
    cst = b.unpack(b.cst)
    small = [q for q, s in enumerate(systems) if s.n == 8 and s.d == 7][:2]
    large = [q for q, s in enumerate(systems) if s.n == 64 and s.d == 31][:1]
    for q in small + large:
        s = systems[q]
        s.cst = cst[q]
        x_ref, _ = oracle.newton(s, items[q][2], int(steps[q]))
        assert np.max(mt.series_rel_error(xs[q], x_ref)) <= cfg.tol, q
    b.close()


def test_batch_flags_singular_and_nonfinite_systems(md):
    """A system whose A_0 has a zero column stops with the singular flag and a
    system started from a NaN stops with the non-finite flag; the others of
    the same launch still converge."""
    items = _mixed(2, 1, SHAPES[:3], 690)
    systems = [s for s, _, _, _ in items]
    x0s = [x0.copy() for _, _, x0, _ in items]
    # system 0: zero the constant coefficient of every monomial containing x_1
    s0 = systems[0]
    s0.coeff = s0.coeff.copy()
    for m in range(s0.M):
        if 1 in s0.vidx[s0.vptr[m]:s0.vptr[m + 1]]:
            s0.coeff[:, :, m, 0] = 0.0
    # system 1: a NaN in the start series
    x0s[1][0, 0, 0, 0] = np.nan
    b = md.Batch(systems)
    x, steps, flags = b.solve(b.pack(x0s), 12, TOL[2])
    assert flags[0] & md.BATCH_SINGULAR
    assert flags[1] & md.BATCH_NONFINITE
    assert flags[2] == md.BATCH_CONVERGED
    x_ref, _ = oracle.newton(systems[2], x0s[2], int(steps[2]))
    assert np.max(mt.series_rel_error(b.unpack(x)[2], x_ref)) <= TOL[2]
    b.close()
