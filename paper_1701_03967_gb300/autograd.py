"""Differentiation through the solver: u = L(a, c)^{-1} f.

L = sum_i a_i 4 h_i^-2 calA_i (x) prod_{j!=i} calC_j + c prod_j calC_j
(Section 4 operator) is symmetric, so for a scalar loss with gradient
g = dloss/du the adjoint solve is the same fast solve: lam = L^{-1} g, and
  dloss/df   = lam,
  dloss/da_i = -lam^T (dL/da_i) u,   dL/da_i = 4 h_i^-2 calA_i (x) prod_{j!=i} calC_j,
  dloss/dc   = -lam^T (dL/dc) u,     dL/dc   = prod_j calC_j,
summed over the right-hand sides.  The two bilinear forms run in the
library's float64 matrix-free apply kernel (fem_fft_grad_coeffs); the solves
run in the plan's precision (mixed: float32 transforms + float64 refinement).
"""

import torch


class FemSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, a, c, plan):
        a_val = tuple(float(x) for x in a.detach().cpu().tolist())
        c_val = float(c.detach().cpu())
        if a_val != tuple(plan.a) or c_val != plan.c:
            plan.set_coefficients(a_val, c_val)
        u = plan.solve(f.detach().contiguous())
        ctx.plan = plan
        ctx.coeffs = (a_val, c_val)
        ctx.save_for_backward(u)
        ctx.a_shape = a.shape
        return u

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        plan = ctx.plan
        a_val, c_val = ctx.coeffs
        if tuple(plan.a) != a_val or plan.c != c_val:
            plan.set_coefficients(a_val, c_val)
        lam = plan.solve(gu.contiguous())
        ga, gc = plan.grad_coeffs(u, lam)
        grad_a = torch.tensor(ga, dtype=torch.float64).reshape(ctx.a_shape)
        grad_c = torch.tensor(gc, dtype=torch.float64)
        return lam, grad_a, grad_c, None


def fem_solve(plan, f, a=None, c=None):
    """u = L(a, c)^{-1} f with gradients for f (CUDA float64 tensor) and the
    CPU float64 tensors a (shape (N,)) and c (scalar).  a, c default to the
    plan's values (then they are constants)."""
    if a is None:
        a = torch.tensor(plan.a, dtype=torch.float64)
    if c is None:
        c = torch.tensor(plan.c, dtype=torch.float64)
    return FemSolve.apply(f, a, c, plan)
