"""torch.autograd binding of the transform: f = Lambda(x) c.

The backward pass is hand-written and runs in the library's kernels:
  * coefficients: grad_c = Lambda^H grad_f (the adjoint transform, sgl_adjoint);
  * points: grad_x_i = Re(conj(grad_f_i) d f_i / d x_i) (window-derivative
    interpolation, sgl_grad_points), with rho held fixed (the factorization
    is exact for every rho >= max |x_i|).
PyTorch's complex convention passes grad_f = dL/dRe f + i dL/dIm f for a real
loss L, for which these are exactly dL/dRe c + i dL/dIm c and dL/dx.
"""
import torch


class NDSGLFT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef, xyz, plan):
        xyz_c = xyz.detach().contiguous()
        coef_c = coef.detach().contiguous()
        plan.set_points(xyz_c)
        f = plan.forward(coef_c)
        ctx.plan = plan
        ctx.save_for_backward(coef_c, xyz_c)
        return f

    @staticmethod
    def backward(ctx, grad_f):
        coef, xyz = ctx.saved_tensors
        plan = ctx.plan
        plan.set_points(xyz)                 # the plan may have served other points since
        g = grad_f.contiguous()
        grad_c = plan.adjoint(g) if ctx.needs_input_grad[0] else None
        grad_x = plan.grad_points(coef, g) if ctx.needs_input_grad[1] else None
        return grad_c, grad_x, None


def ndsglft(coef, xyz, plan):
    """Differentiable forward transform: complex128 [M] values of sum_mu coef_mu H_mu at xyz [M, 3]."""
    return NDSGLFT.apply(coef, xyz, plan)
