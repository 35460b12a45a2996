"""torch.autograd.Functions of the operator with gradients in the links.

DiracFunction: psi -> D[U] psi with gradients in psi and U.

Forward: one stencil apply.  Backward (real loss, torch's convention
grad = dL/dRe + i dL/dIm): grad_psi = D^dagger grad_out, and
grad_U = d Re(grad_out^dagger D[U] psi)/dU from the adjoint kernels (the hops
of Sec. 5.1 and the projection of Sec. 5.2 differentiated exactly).  The
operator is rebuilt from U in forward, so gradients flow to the links used.

InverseActionFunction: (U, phi) -> S = phi^dagger (D^dagger D)^{-1} phi, the
second adjoint quantity; forward runs the two solves once and keeps
dS/dU = -2 d Re(Y^dagger D X)/dU (X = (D^dagger D)^{-1} phi, Y = D X) and
dS/dphi = 2 X (same convention) for backward.
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


class InverseActionFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, phi, op: Brillouin, m0: float, tol: float = 1e-12):
        op.build_hops(U.detach().contiguous())
        dU = torch.zeros_like(U) if ctx.needs_input_grad[0] else None
        S, X, dU, info = op.inverse_action(phi.detach().contiguous(), m0=m0, tol=tol,
                                           want_x=ctx.needs_input_grad[1], dU=dU)
        if info["status"] != "BRI_OK":
            raise RuntimeError("inverse action: solve did not converge: %s" % info)
        ctx.dU, ctx.X = dU, X
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, grad_S):
        grad_U = ctx.dU * grad_S if ctx.dU is not None else None
        grad_phi = 2 * grad_S * ctx.X if ctx.X is not None else None
        return grad_U, grad_phi, None, None, None
