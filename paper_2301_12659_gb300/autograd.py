"""torch.autograd functions over the library's adjoint (real systems).

Tensors here hold multiple double values limb by limb ([K][C][...] float64
arrays, the library's layout), and so do the gradients that flow between
these functions: chain only functions of this module (or others that treat
their inputs as md arrays).  Plain torch arithmetic on such tensors would
treat every limb as an independent double.

    x = NewtonSeries.apply(coeff, nw, x0, steps)   # converged series x(c)
    L = FabryLoss.apply(x, nw)                      # [K] limbs of the loss
    L[0].backward()                                  # coeff.grad: dL/dc (md)

The gradient that reaches FabryLoss is read as one md value dZ/dL (its K
entries the limbs); the backward multiplies dL/dx by it in md on the device
(mdn_md_scale), so a seed such as (3 * L[0]).backward() scales exactly to
the md precision.
"""
import torch


class NewtonSeries(torch.autograd.Function):
    """The series x(c) that Newton's method converges to from x0 for the
    system loaded in `nw` with coefficient series c; its backward is the
    adjoint (mdn_adjoint)."""

    @staticmethod
    def forward(ctx, coeff, nw, x0, steps):
        nw.coeff.copy_(coeff)
        nw.set_series(x0)
        nw.newton(int(steps))
        x = nw.series()
        ctx.nw = nw
        ctx.save_for_backward(x, coeff.detach().clone())
        return x

    @staticmethod
    def backward(ctx, grad_x):
        x, coeff = ctx.saved_tensors
        # the context's coefficients may have been replaced by a later
        # forward: the adjoint needs the Jacobian of this one
        ctx.nw.coeff.copy_(coeff)
        grad = ctx.nw.adjoint(x, grad_x.contiguous())
        return grad, None, None, None


class FabryLoss(torch.autograd.Function):
    """L = sum_i x_{i,d}^2 + x_{0,d-1} / x_{0,d} as [K] limbs (mdn_fabry_loss).
    Backward multiplies dL/dx by the incoming gradient, read as one md value
    (its K entries the limbs), in md on the device (mdn_md_scale)."""

    @staticmethod
    def forward(ctx, x, nw):
        loss, g = nw.fabry_loss(x)
        ctx.nw = nw
        ctx.save_for_backward(g)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (g,) = ctx.saved_tensors
        seed = grad_loss.reshape(g.shape[0], 1).contiguous()  # [K][C=1]
        return ctx.nw.md_scale(seed, g), None
