"""torch.autograd.Function over a CAC-LB rollout: phi_final(theta, sigma).

The forward runs nsteps steps of the CUDA path from a fixed initial state
with the given contact angle of every wall node (degrees, wall-list order)
and surface tension, keeping checkpoints every ckpt_every steps (or, with
outer_every > 0, two-level checkpoints: every outer_every steps, rebuilt
every ckpt_every steps inside each outer segment by the backward); the
backward runs the library's hand-written adjoint and returns dL/dtheta
(FP64-accumulated, per wall node) and dL/dsigma. All arithmetic runs in the
library's kernels; this module only moves tensors across the C ABI.
"""
import torch


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta_wall, sigma, solver, init_phi, init_u, nsteps,
                ckpt_every, outer_every=0):
        solver.set_sigma(float(sigma))
        solver.set_fields(init_phi, init_u)
        solver.set_wall_angles(theta_wall.detach().to("cpu", torch.float32).numpy())
        solver.adjoint_forward(int(nsteps), int(ckpt_every), int(outer_every))
        phi = torch.empty(solver.N, dtype=torch.float32, device="cuda")
        solver.fields_device(phi=phi)
        ctx.solver = solver
        ctx.theta_shape = theta_wall.shape
        ctx.theta_dtype = theta_wall.dtype
        ctx.theta_device = theta_wall.device
        ctx.sigma_dtype = sigma.dtype
        ctx.sigma_device = sigma.device
        return phi.view(solver.shape)

    @staticmethod
    def backward(ctx, grad_phi):
        s = ctx.solver
        g = grad_phi.contiguous().to(torch.float32).view(-1)
        dth = torch.zeros(max(1, ctx.theta_shape[0]), dtype=torch.float64,
                          device="cuda")
        dsg = torch.zeros(1, dtype=torch.float64, device="cuda")
        s.adjoint_backward(g, dth, dsg)
        torch.cuda.current_stream().synchronize()
        dth = dth[:ctx.theta_shape[0]].to(ctx.theta_device, ctx.theta_dtype)
        dsg = dsg[0].to(ctx.sigma_device, ctx.sigma_dtype)
        return dth, dsg, None, None, None, None, None, None


def rollout(theta_wall, sigma, solver, init_phi, init_u=None, nsteps=100,
            ckpt_every=10, outer_every=0):
    """phi after nsteps steps; differentiable in theta_wall and sigma."""
    return Rollout.apply(theta_wall, sigma, solver, init_phi, init_u, nsteps,
                         ckpt_every, outer_every)
