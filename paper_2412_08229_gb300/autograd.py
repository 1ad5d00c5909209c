"""torch.autograd.Functions around unrolled NCO simulations on the GPU.

NCOUnroll: forward runs the C-ABI solver for nsteps with recording (checkpoint every k
steps) and returns the final density and velocity; backward hands their cotangents to
nco_backward, the library's hand-written adjoint, and returns the gradient of the network
parameters. The loss on (rho, u) is ordinary torch code on top.

NCOKineticEnergyUnroll: forward returns the kinetic energy k = (1/2)<|u|^2> after each of
a list of step counts (the library's lbm_kinetic_energy); backward hands dL/dk to
nco_backward_ke. With dissipation_mse below this is the time-dependent training of Sec. IV:
the MSE of -dk/dt against a reference curve.
"""

import torch

from . import lbm_kinetic_energy, lbm_macroscopic, lbm_record_begin, lbm_set_state, lbm_step
from . import nco_backward, nco_backward_ke, nco_set_weights


class NCOUnroll(torch.autograd.Function):
    """rho, u = NCOUnroll.apply(theta, ctx, f0, nsteps, k).

    theta: (1064,) or (1484,) float32 CUDA tensor (requires_grad); ctx: an lbm context
    created with op="nco", storage="f32", net="f32"; f0: (27, nz, ny, nx) float32 CUDA
    tensor of initial populations (not differentiated here; its cotangent is available
    from nco_backward). A forced context needs the random draws of its nsteps steps queued
    (lbm_force_draws) before each call; each step's force enters as an input of the step.
    One recording per context: call backward before the next forward on the same context.
    """

    @staticmethod
    def forward(fctx, theta, lbm_ctx, f0, nsteps, k):
        nco_set_weights(lbm_ctx, theta.detach().contiguous())
        lbm_set_state(lbm_ctx, f0.detach().contiguous())
        lbm_record_begin(lbm_ctx, k)
        lbm_step(lbm_ctx, nsteps)
        shape = lbm_ctx.shape
        rho = torch.empty(shape, device=theta.device, dtype=torch.float32)
        u = torch.empty((3,) + shape, device=theta.device, dtype=torch.float32)
        lbm_macroscopic(lbm_ctx, rho, u)
        fctx.lbm_ctx = lbm_ctx
        fctx.ntheta = int(theta.numel())
        return rho, u

    @staticmethod
    def backward(fctx, d_rho, d_u):
        dev = d_u.device if d_u is not None else d_rho.device
        dtheta = torch.empty(fctx.ntheta, device=dev, dtype=torch.float32)
        nco_backward(fctx.lbm_ctx,
                     None if d_u is None else d_u.contiguous().float(),
                     None if d_rho is None else d_rho.contiguous().float(),
                     dtheta, None)
        return dtheta, None, None, None, None


class NCOKineticEnergyUnroll(torch.autograd.Function):
    """ke = NCOKineticEnergyUnroll.apply(theta, ctx, f0, obs_steps, k).

    obs_steps: increasing step counts (0 allowed); ke: float64 CUDA tensor of
    k = (1/2)<|u|^2> after each. ctx, theta and f0 as for NCOUnroll (any boundary the
    adjoint covers, e.g. the reduced Taylor-Green domain).
    """

    @staticmethod
    def forward(fctx, theta, lbm_ctx, f0, obs_steps, k):
        steps = [int(s) for s in obs_steps]
        if any(b < a for a, b in zip(steps, steps[1:])) or (steps and steps[0] < 0):
            raise ValueError("obs_steps must be non-negative and increasing")
        nco_set_weights(lbm_ctx, theta.detach().contiguous())
        lbm_set_state(lbm_ctx, f0.detach().contiguous())
        lbm_record_begin(lbm_ctx, k)
        ke = torch.empty(len(steps), device=theta.device, dtype=torch.float64)
        t = 0
        for j, s in enumerate(steps):
            if s > t:
                lbm_step(lbm_ctx, s - t)
                t = s
            lbm_kinetic_energy(lbm_ctx, ke[j:j + 1])
        fctx.lbm_ctx = lbm_ctx
        fctx.steps = steps
        fctx.ntheta = int(theta.numel())
        return ke

    @staticmethod
    def backward(fctx, d_ke):
        dtheta = torch.empty(fctx.ntheta, device=d_ke.device, dtype=torch.float32)
        nco_backward_ke(fctx.lbm_ctx, fctx.steps, d_ke.detach().double().cpu().numpy(), dL_dtheta=dtheta)
        return dtheta, None, None, None, None


def dissipation_rate(ke, dt):
    """-dk/dt by central differences of a uniformly sampled k (interior samples)."""
    return -(ke[2:] - ke[:-2]) / (2.0 * dt)


def dissipation_mse(ke, dt, eps_ref):
    """Sec. IV's loss: the mean squared difference of -dk/dt from the reference eps_ref
    at the interior samples (k sampled every dt, len(eps_ref) + 2 samples)."""
    d = dissipation_rate(ke, dt) - eps_ref
    return (d * d).mean()
