"""torch.autograd.Function for the implicit heat step objective.

J(P, r, x0, y0, k_q) = 1/2 int_box (theta_h - theta*_h)^2 after one backward-Euler heat step
driven by the Gaussian laser flux of eq. (laser_gauss), with a per-Gauss-point conductivity
field k_q.  The forward pass calls mf_heat_step_gradient, which solves the forward system,
the adjoint system A^T lambda = dJ/dtheta and forms dJ/dp = lambda^T df/dp and
dJ/dk_q = -w_q |J| grad(lambda) . grad(theta) in the library's kernels; backward only scales
those gradients by the incoming gradient.
"""
import torch


class HeatStepObjective(torch.autograd.Function):

    @staticmethod
    def forward(ctx, laser, kq, op, theta_prev, theta_target, box_half, box_depth, absorptivity, solver_kw):
        """laser: fp64 tensor (P, r, x0, y0); kq: fp64 CUDA tensor of n_cells * 27 values."""
        op.set_field("k_qpoint", kq.detach().contiguous())
        p = [float(v) for v in laser.detach().cpu().tolist()] + [float(absorptivity)]
        J, g, gk, _, _ = op.heat_step_gradient(p, theta_prev, theta_target, box_half, box_depth,
                                               with_kq=True, **(solver_kw or {}))
        ctx.save_for_backward(torch.tensor(g, dtype=torch.float64, device=laser.device), gk)
        return torch.tensor(J, dtype=torch.float64, device=laser.device)

    @staticmethod
    def backward(ctx, grad_out):
        g, gk = ctx.saved_tensors
        return (grad_out * g, grad_out.to(gk.device) * gk, None, None, None, None, None, None, None)


def heat_step_objective(op, laser, kq, theta_prev, theta_target, box_half, box_depth, absorptivity=0.35,
                        **solver_kw):
    return HeatStepObjective.apply(laser, kq, op, theta_prev, theta_target, box_half, box_depth, absorptivity,
                                   solver_kw)
