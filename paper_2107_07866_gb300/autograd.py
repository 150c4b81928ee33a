"""torch.autograd wrapper of the knot-gradient kernels (potential fitting).

loss = eam_loss(knots, sim, Fref, Eref) evaluates, on the GPU, the
force-matching + energy loss of sim's current configuration(s) for the
spline knot values ``knots`` (a (3, n) float64 tensor: f, phi, F) and
returns a 0-d tensor whose backward gives d loss / d knots from the
hand-written adjoint kernels (misa_loss_grad).  Argument marshalling only.
"""
from __future__ import annotations

import torch


class EAMLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, knots, sim, Fref, Eref):
        k = knots.detach().to(torch.float64).contiguous()
        if k.is_cuda:
            sim.set_tables(k[0], k[1], k[2])
            grad = torch.empty(k.numel(), dtype=torch.float64, device=k.device)
        else:
            kn = k.numpy()
            sim.set_tables(kn[0], kn[1], kn[2])
            grad = torch.empty(k.numel(), dtype=torch.float64)
        loss, _ = sim.loss_grad(Fref, Eref, grad=grad if k.is_cuda else grad.numpy())
        ctx.save_for_backward(grad.reshape(k.shape).to(knots.dtype))
        return knots.new_tensor(loss)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None


def eam_loss(knots, sim, Fref, Eref):
    return EAMLoss.apply(knots, sim, Fref, Eref)
