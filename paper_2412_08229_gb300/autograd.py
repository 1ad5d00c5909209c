"""torch.autograd.Function around an unrolled NCO simulation on the GPU.

Forward runs the C-ABI solver for nsteps with recording (checkpoint every k steps) and
returns the final density and velocity; backward hands their cotangents to
nco_backward, the library's hand-written adjoint, and returns the gradient of the
network parameters. The loss on (rho, u) is ordinary torch code on top.
"""

import torch

from . import lbm_get_state, lbm_macroscopic, lbm_record_begin, lbm_set_state, lbm_step
from . import nco_backward, nco_set_weights


class NCOUnroll(torch.autograd.Function):
    """rho, u = NCOUnroll.apply(theta, ctx, f0, nsteps, k).

    theta: (1064,) float32 CUDA tensor (requires_grad); ctx: an lbm context created with
    op="nco", storage="f32", net="f32"; f0: (27, nz, ny, nx) float32 CUDA tensor of initial
    populations (not differentiated here; its cotangent is available from nco_backward).
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
        return rho, u

    @staticmethod
    def backward(fctx, d_rho, d_u):
        dtheta = torch.empty(1064, device=d_u.device if d_u is not None else d_rho.device, dtype=torch.float32)
        nco_backward(fctx.lbm_ctx,
                     None if d_u is None else d_u.contiguous().float(),
                     None if d_rho is None else d_rho.contiguous().float(),
                     dtheta, None)
        return dtheta, None, None, None, None
