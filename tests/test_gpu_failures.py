"""Failure detection of the GPU path, tested without a GPU fault: every
condition the library detects comes back as a status code through the C-ABI
and leaves the context usable.

* A bounded device wait that runs out: the wait limit of the dataflow
  kernels (QR of A0, forward substitution) is lowered to 1 microsecond, far
  below one column period of the QR, so the waits give up, record the
  timeout and return; mdn_newton reports MDN_ETIMEOUT.  With the default
  limit restored the same context runs Newton to the oracle's result.
* Early stopping (mdn_newton with tol > 0, the stopping test of the
  problem statement of Section 2) and MDN_ENOTCONVERGED with the series
  still readable.
"""
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


def test_wait_limit_runs_out_and_context_recovers(md):
    cfg = wl.small_config(4, 1, n=64, d=7, mono_per_eq=2, kmin=1, kmax=3, steps=6, index=520)
    s, xstar, x0 = planted(cfg)
    nw = md.Newton(s)
    nw.set_wait_limit_ns(1000)
    nw.set_series(x0)
    with pytest.raises(md.MdnError) as e:
        nw.newton(2)
    assert e.value.status == md.MDN_ETIMEOUT
    with pytest.raises(md.MdnError) as e:
        nw.set_wait_limit_ns(0)
    assert e.value.status == md.MDN_EINVAL
    nw.set_wait_limit_ns(2_000_000_000)
    nw.set_series(x0)
    nw.newton(cfg.steps)
    x_ref, _ = oracle.newton(s, x0, cfg.steps)
    assert np.max(mt.series_rel_error(to_np(nw.series()), x_ref)) <= cfg.tol


def test_newton_stops_early_at_the_tolerance(md):
    """tol > 0: the loop ends after the first step with ||dx||_1 <= tol; the
    series is that of the oracle after the same number of steps."""
    cfg = wl.small_config(2, 1, n=6, d=9, mono_per_eq=3, kmin=1, kmax=3, steps=12, index=521)
    s, xstar, x0 = planted(cfg)
    nw = md.Newton(s)
    nw.set_series(x0)
    hist = nw.newton(12, tol=1e-20)
    done = nw.steps_done
    assert 1 <= done < 12 and len(hist) == done
    assert hist[-1, 2] <= 1e-20 and np.all(hist[:-1, 2] > 1e-20)
    x_ref, h_ref = oracle.newton(s, x0, done)
    assert np.max(mt.series_rel_error(to_np(nw.series()), x_ref)) <= cfg.tol
    assert np.max(mt.series_rel_error(to_np(nw.series()), xstar)) <= 1e-18


def test_newton_reports_not_converged(md):
    """Two steps from 1e-3 noise cannot reach ||dx||_1 <= 1e-60: the call
    returns MDN_ENOTCONVERGED after max_steps, and x is the two-step series."""
    cfg = wl.small_config(4, 1, n=5, d=9, mono_per_eq=3, kmin=1, kmax=3, steps=2, index=522)
    s, xstar, x0 = planted(cfg)
    nw = md.Newton(s)
    nw.set_series(x0)
    with pytest.raises(md.MdnError) as e:
        nw.newton(2, tol=1e-60)
    assert e.value.status == md.MDN_ENOTCONVERGED
    assert nw.steps_done == 2
    x_ref, _ = oracle.newton(s, x0, 2)
    assert np.max(mt.series_rel_error(to_np(nw.series()), x_ref)) <= cfg.tol
