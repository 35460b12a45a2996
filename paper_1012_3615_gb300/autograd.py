"""torch.autograd.Function for psi -> D[U] psi with gradients in psi and U.

Forward: one stencil apply.  Backward (real loss, torch's convention
grad = dL/dRe + i dL/dIm): grad_psi = D^dagger grad_out, and
grad_U = d Re(grad_out^dagger D[U] psi)/dU from the adjoint kernels (the hops
of Sec. 5.1 and the projection of Sec. 5.2 differentiated exactly).  The
operator is rebuilt from U in forward, so gradients flow to the links used.
"""
import torch

from .core import Brillouin


class DiracFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, psi, op: Brillouin, m0: float):
        op.build_hops(U.detach().contiguous())
        out = op.apply(psi.detach().contiguous(), m0=m0)
        ctx.save_for_backward(psi)
        ctx.op = op
        ctx.m0 = m0
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (psi,) = ctx.saved_tensors
        op, m0 = ctx.op, ctx.m0
        g = grad_out.contiguous()
        grad_U = grad_psi = None
        if ctx.needs_input_grad[1]:
            grad_psi = op.apply(g, m0=m0, dagger=True)
        if ctx.needs_input_grad[0]:
            grad_U = op.force(g, psi.detach().contiguous(), m0=m0)
        return grad_U, grad_psi, None, None
