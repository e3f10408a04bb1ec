"""torch.autograd.Function over the stage residual (tangent and adjoint kernels).

Forward: R(k; tau, u) (lh_residual).  Reverse mode: grad_k = J^T grad_R (lh_jtvp,
hand-written adjoint of the quadrature-point kernel).  Forward mode: J dk (lh_jvp).
Gradients flow to k only (u and tau are treated as constants); quadrature-point state
is recomputed inside each kernel rather than stored.
"""
import torch


class StageResidual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, k, u, tau, mesh):
        ctx.mesh, ctx.tau = mesh, float(tau)
        ctx.save_for_backward(k, u)
        ctx.save_for_forward(k, u)
        return mesh.residual(u.detach(), k.detach(), tau)

    @staticmethod
    def backward(ctx, grad_r):
        k, u = ctx.saved_tensors
        g = ctx.mesh.jtvp(u.detach(), k.detach(), ctx.tau, grad_r.contiguous())
        return g, None, None, None

    @staticmethod
    def jvp(ctx, dk, du, dtau, dmesh):
        k, u = ctx.saved_tensors
        if dk is None:
            return torch.zeros_like(k)
        return ctx.mesh.jvp(u.detach(), k.detach(), ctx.tau, dk.contiguous())
