"""The pseudofermion action S_f = phi^dag (M^dag M)^{-1} phi as a torch.autograd.Function.

Forward solves M^dag M X = phi and reduces phi^dag X in the CUDA library;
backward recomputes X (it is not stored), then the library's adjoint
kernel returns dS_f / dU in torch's complex-gradient convention, and
dS_f / dphi = 2 X.  Every step runs in the library; this module only
passes tensors through the C interface.
"""
import torch

from . import lq


class PseudofermionAction(torch.autograd.Function):
    """S_f(U, phi) for U complex128 (V, 4, 3, 3) and phi complex128 (V, 4, 3) on the GPU."""

    @staticmethod
    def forward(fctx, U, phi, dims, kappa, tol, inner_prec, t_antiperiodic):
        U = U.contiguous()
        phi = phi.contiguous()
        ctx = lq.lq_create(dims, t_antiperiodic)
        try:
            lq.lq_gauge_set(ctx, U)
            S = lq.lq_pseudofermion_action(ctx, phi, kappa, tol, 100000, inner_prec)
        finally:
            lq.lq_destroy(ctx)
        fctx.save_for_backward(U, phi)
        fctx.args = (dims, kappa, tol, inner_prec, t_antiperiodic)
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(fctx, gS):
        U, phi = fctx.saved_tensors
        dims, kappa, tol, inner_prec, t_antiperiodic = fctx.args
        ctx = lq.lq_create(dims, t_antiperiodic)
        try:
            lq.lq_gauge_set(ctx, U)
            X = torch.empty_like(phi)
            lq.lq_solve_MdagM(ctx, X, phi, kappa, tol, 100000, inner_prec, 50)
            G = torch.empty_like(U)
            lq.lq_fermion_grad(ctx, G, X, kappa)
        finally:
            lq.lq_destroy(ctx)
        g = gS.to(torch.float64)
        gU = G * g if fctx.needs_input_grad[0] else None
        gphi = 2.0 * X * g if fctx.needs_input_grad[1] else None
        return gU, gphi, None, None, None, None, None


def pseudofermion_action(U, phi, dims, kappa, tol=1e-10, inner_prec=lq.LQ_F64, t_antiperiodic=True):
    """Differentiable S_f = phi^dag (M^dag M)^{-1} phi."""
    return PseudofermionAction.apply(U, phi, tuple(dims), float(kappa), float(tol), int(inner_prec),
                                     bool(t_antiperiodic))
