"""Helpers of the GPU parity tests: run the CUDA library and the oracle on the same inputs."""

import numpy as np

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from oracle import stepper as S


def torch_cuda():
    import torch
    return torch


def to_oracle_f(f_soa):
    """(27, nz, ny, nx) -> (nz, ny, nx, 27) float64."""
    return np.moveaxis(np.asarray(f_soa, dtype=np.float64), 0, -1)


def to_soa_f(f_aos):
    return np.ascontiguousarray(np.moveaxis(f_aos, -1, 0)).astype(np.float32)


def make_ctx(shape, nu, op, storage="f32", net="f32", bc="periodic", theta=None, forcing=None):
    nz, ny, nx = shape
    ctx = P.lbm_create(nx, ny, nz, nu, op=op, storage=storage, net=net, boundary=bc, forcing=forcing)
    if op == "nco":
        P.nco_set_weights(ctx, np.asarray(theta, dtype=np.float32))
    return ctx


def gpu_state(ctx):
    torch = torch_cuda()
    f = torch.empty((27,) + ctx.shape, dtype=torch.float32, device="cuda")
    P.lbm_get_state(ctx, f)
    torch.cuda.synchronize()
    return f.cpu().numpy()


def set_gpu_state(ctx, f_soa):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(f_soa, dtype=np.float32)).cuda()
    P.lbm_set_state(ctx, t)
    torch.cuda.synchronize()


def init_gpu(ctx, rho, u):
    torch = torch_cuda()
    r = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32)).cuda()
    v = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
    P.lbm_init(ctx, r, v)
    torch.cuda.synchronize()


def oracle_sim_from_fields(rho, u, tau, op, theta=None, bc="periodic", forcing=None, sizes=col.LAYER_SIZES):
    """Oracle started from the FP32-rounded fields the GPU receives."""
    rho32 = np.asarray(rho, dtype=np.float32).astype(np.float64)
    u32 = np.moveaxis(np.asarray(u, dtype=np.float32).astype(np.float64), 0, -1)
    th = None if theta is None else np.asarray(theta, dtype=np.float32).astype(np.float64)
    return S.Simulation.from_macroscopic(rho32, u32, tau, op=op, theta=th, bc=bc, forcing=forcing, sizes=sizes)


def rel_maxnorm(a, ref):
    return float(np.abs(np.asarray(a, np.float64) - ref).max() / np.abs(ref).max())


def theta0():
    return lbm_inputs.nco_parameters(0).astype(np.float32)


def check_bf16_step(ctx, nu, theta, sizes=col.LAYER_SIZES, bc="periodic", storage="f32"):
    """Step a BF16-network context once from its current state and check every stored
    population against the BF16-operand oracle and its bound (tests/bf16_ref.py)."""
    from tests import bf16_ref as B
    start = to_oracle_f(gpu_state(ctx))
    P.lbm_step(ctx, 1)
    assert P.lbm_check(ctx) == 0
    got = to_oracle_f(gpu_state(ctx))
    ref, bound = B.step_reference(start, col.tau_from_nu(nu), np.asarray(theta, np.float64), sizes, bc)
    ok = B.within(got, ref, bound, storage)
    assert ok.all(), (f"{(~ok).sum()} of {ok.size} populations outside the BF16 bound; "
                      f"max |got - ref| {np.abs(got - ref).max():.3e}")
