"""Pins of the oracle's staggered Newton with the QR of A_0 once
(Sections 4 and 5.3): the order schedule, the untouched higher coefficients,
the order-1 phase as plain Newton on x_0 alone, and recovery of planted
solutions."""
import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import metrics as mt


def test_order_schedule():
    cfg = wl.small_config(2, 1, n=3, d=31, mono_per_eq=2, kmin=1, kmax=3, index=540)
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    _, _, orders = oracle.newton_staggered(s, x0, 12, 3)
    # L := L + 1 + L/2 from L = 1 after three order-1 steps, capped at d+1 = 32
    assert orders.tolist() == [1, 1, 1, 2, 4, 7, 11, 17, 26, 32, 32, 32]


def test_higher_coefficients_untouched_and_order_one_is_newton_on_x0():
    cfg = wl.small_config(4, 1, n=4, d=9, mono_per_eq=3, kmin=1, kmax=3, index=541)
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    x3, h3, orders = oracle.newton_staggered(s, x0, 3, 3)
    assert np.all(orders == 1)
    assert np.array_equal(x3[..., 1:], x0[..., 1:])
    # order 1 is the system mod t: plain Newton on the constant coefficients
    s0 = wl.System(s.K, s.C, s.n, 0, s.eq, s.vptr, s.vidx, s.coeff[..., :1].copy(), s.cst[..., :1].copy())
    xp, hp = oracle.newton(s0, x0[..., :1].copy(), 3)
    assert np.array_equal(x3[..., :1], xp)
    assert np.array_equal(h3, hp)
    x5, _, orders = oracle.newton_staggered(s, x0, 5, 3)
    assert orders.tolist() == [1, 1, 1, 2, 4]
    assert np.array_equal(x5[..., 4:], x0[..., 4:])


@pytest.mark.parametrize("K,C,first,steps", [(2, 1, 4, 12), (4, 1, 5, 14), (8, 2, 6, 15)])
def test_staggered_recovers_plant(K, C, first, steps):
    cfg = wl.small_config(K, C, n=4, d=15, mono_per_eq=3, kmin=1, kmax=3, index=542 + K)
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    x, hist, orders = oracle.newton_staggered(s, x0, steps, first)
    assert orders[-1] == 16
    assert np.max(mt.series_rel_error(x, xstar)) <= cfg.tol
