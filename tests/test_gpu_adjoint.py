"""The adjoint through the C-ABI (mdn_adjoint, mdn_fabry_loss) and the
torch.autograd functions over it: gradients of the Fabry-ratio loss of the
converged series with respect to every coefficient series, against the
oracle's adjoint (itself pinned to octo double central differences) and,
at full size, against octo double central differences taken with the
library's own octo double Newton (an independent code path: the forward
solver), to the relative tolerance 1e-24."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import oracle
from paper_2301_12659_gb300 import workloads as wl
from tests import exact as ex
from tests import metrics as mt
from tests.gpu_util import need_gpu, planted, to_np

pytestmark = pytest.mark.gpu
REL = 1e-24


@pytest.fixture(scope="module")
def md():
    return need_gpu()


def _close(got, ref, rel=REL):
    """|got - ref| <= rel * max(|ref|, 1e-6 max|ref|) entry by entry."""
    err = mt.magnitude(mt.md_diff(got, ref))
    val = mt.magnitude(mt.md_value(ref))
    den = np.maximum(val, 1e-6 * np.max(val))
    return float(np.max(err / den))


@pytest.mark.parametrize("n,d,index", [(3, 5, 530), (9, 15, 531), (33, 31, 532)])
def test_adjoint_matches_oracle(md, n, d, index):
    cfg = wl.small_config(2, 1, n=n, d=d, mono_per_eq=3, kmin=1, kmax=5, steps=8, index=index)
    s, xstar, x0 = planted(cfg)
    nw = md.Newton(s)
    nw.set_series(x0)
    nw.newton(cfg.steps)
    x = nw.series()
    loss, g = nw.fabry_loss(x)
    L_ref, g_ref = oracle.fabry_loss(to_np(x))
    assert abs(ex.md_to_fr(to_np(loss)) - ex.md_to_fr(L_ref)) <= abs(ex.md_to_fr(L_ref)) * Fr(2) ** -100
    assert _close(to_np(g), g_ref) <= 1e-30
    grad = to_np(nw.adjoint(x, g))
    grad_ref = oracle.adjoint(s, to_np(x), g_ref)
    assert _close(grad, grad_ref) <= REL


def test_autograd_functions(md):
    import torch
    from paper_2301_12659_gb300.autograd import FabryLoss, NewtonSeries
    cfg = wl.small_config(2, 1, n=6, d=11, mono_per_eq=3, kmin=1, kmax=4, steps=8, index=533)
    s, xstar, x0 = planted(cfg)
    nw = md.Newton(s)
    coeff = nw.coeff.clone().requires_grad_(True)
    x0d = torch.as_tensor(x0, device=coeff.device)
    x = NewtonSeries.apply(coeff, nw, x0d, cfg.steps)
    L = FabryLoss.apply(x, nw)
    L[0].backward()
    L_ref, g_ref = oracle.fabry_loss(to_np(x.detach()))
    grad_ref = oracle.adjoint(s, to_np(x.detach()), g_ref)
    assert _close(to_np(coeff.grad), grad_ref) <= REL
    assert abs(float(L[0].detach()) - L_ref[0]) <= 1e-15 * abs(L_ref[0])


def test_autograd_upstream_gradient_is_applied_in_md(md):
    """A seed that is not a power of two ((L[0] / 3).backward(): the
    incoming gradient is the double 1/3) scales dL/dc in md on the device:
    the gradient is the oracle's adjoint of the exact scaled g, to 1e-24.
    Two forwards before the backwards: each graph keeps the coefficients of
    its own forward."""
    import torch
    from paper_2301_12659_gb300.autograd import FabryLoss, NewtonSeries
    cfg = wl.small_config(2, 1, n=6, d=11, mono_per_eq=3, kmin=1, kmax=4, steps=8, index=534)
    s, xstar, x0 = planted(cfg)
    nw = md.Newton(s)
    x0d = torch.as_tensor(x0, device=nw.coeff.device)
    c1 = nw.coeff.clone().requires_grad_(True)
    x1 = NewtonSeries.apply(c1, nw, x0d, cfg.steps)
    L1 = FabryLoss.apply(x1, nw)
    # a second forward on the same context with other coefficients
    c2_np = s.coeff.copy()
    c2_np[:, :, 0, 3] *= 0.5
    c2 = torch.as_tensor(c2_np, device=nw.coeff.device).requires_grad_(True)
    x2 = NewtonSeries.apply(c2, nw, x0d, cfg.steps)
    L2 = FabryLoss.apply(x2, nw)
    (L1[0] / 3.0).backward()
    L2[0].backward()
    third = Fr(1, 3)
    seed = float(third)  # the double the division hands down
    for c, x, coeff_np in ((c1, x1, s.coeff), (c2, x2, c2_np)):
        sc = wl.System(s.K, s.C, s.n, s.d, s.eq, s.vptr, s.vidx, coeff_np, s.cst)
        _, g_ref = oracle.fabry_loss(to_np(x.detach()))
        grad_ref = oracle.adjoint(sc, to_np(x.detach()), g_ref)
        if c is c1:
            grad_ref = oracle.md_binary("mul", grad_ref.reshape(s.K, 1, -1),
                                        np.broadcast_to(np.array([seed] + [0.0] * (s.K - 1)).reshape(s.K, 1, 1),
                                                        (s.K, 1, grad_ref[0, 0].size))).reshape(grad_ref.shape)
        assert _close(to_np(c.grad), grad_ref) <= REL


def _promote(a, K=8):
    out = np.zeros((K,) + a.shape[1:])
    out[:a.shape[0]] = a
    return out


def test_adjoint_workload_against_octo_double_central_differences(md):
    """dd, n = 64, d = 31: the adjoint gradient against (L(c+hu) - L(c-hu))/2h
    with L from the library's octo double Newton on the exactly promoted
    system (h = 1e-20), for 8 random +-1 directions and 32 single
    coefficients; and against the oracle's adjoint entry by entry."""
    import torch
    cfg = wl.ADJOINT_CONFIG
    s, xstar, x0 = planted(cfg)
    nw = md.Newton(s)
    nw.set_series(x0)
    nw.newton(cfg.steps)
    x = nw.series()
    loss, g = nw.fabry_loss(x)
    grad = to_np(nw.adjoint(x, g))
    grad_ref = oracle.adjoint(s, to_np(x), oracle.fabry_loss(to_np(x))[1])
    assert _close(grad, grad_ref) <= REL
    # octo double forward solves
    s8 = wl.System(8, 1, s.n, s.d, s.eq, s.vptr, s.vidx, _promote(s.coeff), _promote(s.cst))
    n8 = md.Newton(s8)
    x8_start = torch.as_tensor(_promote(to_np(x)), device=x.device)
    base = n8.coeff.clone()
    h = Fr(1e-20)

    def loss_od(delta):  # delta: dict (m, j) -> Fraction shift
        c = base.clone().cpu().numpy()
        for (m, j), dv in delta.items():
            c[:, 0, m, j] = ex.fr_to_md(ex.md_to_fr(c[:, 0, m, j]) + dv, 8)
        n8.coeff.copy_(torch.as_tensor(c, device=x.device))
        n8.set_series(x8_start)
        n8.newton(4)
        L8, _ = n8.fabry_loss(n8.series())
        return ex.md_to_fr(to_np(L8))

    rng = np.random.default_rng(7)
    scale = float(np.max(np.abs(grad[0, 0])))
    for _ in range(32):
        m, j = int(rng.integers(s.M)), int(rng.integers(s.D))
        fd = (loss_od({(m, j): h}) - loss_od({(m, j): -h})) / (2 * h)
        adj = ex.md_to_fr(grad[:, 0, m, j])
        assert abs(fd - adj) <= Fr(REL) * max(abs(adj), Fr(1e-6) * Fr(scale)), (m, j, float(fd), float(adj))
    for _ in range(8):
        u = rng.choice([-1, 1], size=(s.M, s.D))
        plus = {(m, j): h * int(u[m, j]) for m in range(s.M) for j in range(s.D)}
        minus = {k: -v for k, v in plus.items()}
        fd = (loss_od(plus) - loss_od(minus)) / (2 * h)
        adj = Fr(0)
        for m in range(s.M):
            for j in range(s.D):
                adj += ex.md_to_fr(grad[:, 0, m, j]) * int(u[m, j])
        assert abs(fd - adj) <= Fr(REL) * abs(adj)
