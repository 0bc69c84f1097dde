"""dJ/dkappa behind ``torch.autograd.Function``.

forward: sets kappa on the hierarchy, solves A(kappa) u = b with GMG-PCG and
returns J = (u - u_d)^T M (u - u_d); only the fine-level u is kept
(checkpoint).  backward: one adjoint solve A lambda = -2 M (u - u_d) from the
checkpoint plus the fused per-cell kernel g_K = int_K grad(lambda).grad(u).
All arithmetic runs in the CUDA library (fe_solve_poisson, fe_objective,
fe_adjoint_gradient).
"""
import torch

from . import FE_RHS_NODAL_F, default_opts


class PoissonObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, hier, rhs, u_d, rhs_kind=FE_RHS_NODAL_F, opts=None):
        o = opts if opts is not None else default_opts(rtol=1e-12)
        kappa_c = kappa.detach().contiguous().to(torch.float64)
        hier.set_coefficient(kappa_c)
        u = torch.empty(hier.n_dofs(), dtype=torch.float64, device=kappa.device)
        hier.solve(rhs, u, rhs_kind=rhs_kind, opts=o)
        J = hier.objective(u, u_d)
        ctx.hier, ctx.rhs, ctx.u_d, ctx.rhs_kind, ctx.opts = hier, rhs, u_d, rhs_kind, o
        ctx.save_for_backward(u, kappa_c)
        return torch.tensor(J, dtype=torch.float64, device=kappa.device)

    @staticmethod
    def backward(ctx, grad_out):
        u, kappa_c = ctx.saved_tensors
        hier = ctx.hier
        hier.set_coefficient(kappa_c)  # the hierarchy may have been reused since forward
        g = torch.empty(hier.n_cells(), dtype=torch.float64, device=u.device)
        hier.adjoint_gradient(ctx.rhs, ctx.u_d, g, rhs_kind=ctx.rhs_kind, u_ckpt=u, opts=ctx.opts)
        return grad_out * g, None, None, None, None, None


def poisson_objective(kappa, hier, rhs, u_d, rhs_kind=FE_RHS_NODAL_F, opts=None):
    """J(kappa) = int (u_h(kappa) - I_h u_d)^2, differentiable in kappa (per fine cell)."""
    return PoissonObjective.apply(kappa, hier, rhs, u_d, rhs_kind, opts)
