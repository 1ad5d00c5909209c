"""GPU tests of the adjoint for the time-dependent training of Sec. IV: the three-hidden-
layer network, the reduced Taylor-Green domain of Appendix A, and kinetic-energy
observations (nco_backward_ke) driving the dissipation-rate loss, each against autograd of
the FP64 PyTorch restatement of the oracle (itself pinned by central differences of the
NumPy oracle on the CPU).

Tolerance: 1e-3 relative in the 2-norm (FP32 adjoint against FP64 references), as for the
two-hidden-layer adjoint; the same gradient for any checkpoint interval to 1e-6.
"""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from oracle import diagnostics as D
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from oracle import torch_ref as T  # noqa: E402

DEEP = (27, 20, 20, 20, 4)
SHALLOW = (27, 20, 20, 4)
NU = 0.004


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def _theta(sizes, seed=0):
    return lbm_inputs.nco_parameters(seed, sizes).astype(np.float32).astype(np.float64)


def _start(n, bc):
    """FP32-rounded equilibrium start: the reduced Taylor-Green domain's corner of the
    shifted-grid vortex, or the mirror octant."""
    if bc == "tgv_reduced":
        rho, u = lbm_inputs.taylor_green_3d(4 * n, 0.05, shifted=True)
        rho, u = rho[:n, :n, :n], u[:, :n, :n, :n]
    elif bc == "periodic":
        rho, u = lbm_inputs.taylor_green_3d(n, 0.05)
    else:
        rho, u = lbm_inputs.taylor_green_octant(n, 0.05)
    f0 = col.equilibrium(rho, np.moveaxis(u, 0, -1))
    return f0.astype(np.float32).astype(np.float64)


def _ctx(n, bc, theta):
    ctx = G.make_ctx((n, n, n), NU, "nco", bc=bc, theta=theta.astype(np.float32))
    return ctx


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _quadratic_reference(f0, theta, nsteps, bc, sizes):
    th = torch.tensor(theta, requires_grad=True)
    f0t = torch.tensor(f0, requires_grad=True)
    f = T.run(f0t, col.tau_from_nu(NU), th, nsteps, bc=bc, sizes=sizes)
    loss = (T.velocity(f) ** 2).sum() + ((f.sum(-1) - 1.0) ** 2).sum()
    loss.backward()
    return th.grad.numpy(), f0t.grad.numpy()


def _quadratic_gpu(f0, theta, nsteps, bc, k):
    n = f0.shape[0]
    ctx = _ctx(n, bc, theta)
    G.set_gpu_state(ctx, np.moveaxis(f0, -1, 0))
    P.lbm_record_begin(ctx, k)
    P.lbm_step(ctx, nsteps)
    rho = torch.empty((n, n, n), device="cuda")
    u = torch.empty((3, n, n, n), device="cuda")
    P.lbm_macroscopic(ctx, rho, u)
    du = (2.0 * u).contiguous()
    drho = (2.0 * (rho - 1.0)).contiguous()
    dtheta = torch.zeros(theta.size, device="cuda")
    df0 = torch.zeros((27, n, n, n), device="cuda")
    P.nco_backward(ctx, du, drho, dtheta, df0)
    torch.cuda.synchronize()
    return dtheta.cpu().numpy().astype(np.float64), np.moveaxis(df0.cpu().numpy(), 0, -1).astype(np.float64)


@pytest.mark.parametrize("bc,sizes", [("mirror", DEEP), ("tgv_reduced", SHALLOW), ("tgv_reduced", DEEP),
                                      ("periodic", DEEP)])
def test_adjoint_matches_autograd_reference(bc, sizes):
    n = 4 if bc == "tgv_reduced" else 6
    f0 = _start(n, bc)
    theta = _theta(sizes)
    g_ref, gf_ref = _quadratic_reference(f0, theta, 6, bc, sizes)
    g_gpu, gf_gpu = _quadratic_gpu(f0, theta, 6, bc, k=4)
    assert g_gpu.size == theta.size
    assert _rel(g_gpu, g_ref) <= 1e-3
    assert _rel(gf_gpu, gf_ref) <= 1e-3


def _obs(every, nsamples):
    return [every * j for j in range(nsamples + 2)]


def _eps_ref(f0, theta, obs, dt, sizes):
    """A synthetic reference dissipation curve: half the restatement's own (the paper's
    512^3 DNS curve is not available)."""
    with torch.no_grad():
        ke = T.run_kinetic_energy(torch.tensor(f0), col.tau_from_nu(NU), torch.tensor(theta), obs,
                                  bc="tgv_reduced", sizes=sizes).numpy()
    return 0.5 * D.dissipation(ke, dt)


def _dissipation_reference(f0, theta, obs, dt, eps_ref, sizes):
    th = torch.tensor(theta, requires_grad=True)
    ke = T.run_kinetic_energy(torch.tensor(f0), col.tau_from_nu(NU), th, obs, bc="tgv_reduced", sizes=sizes)
    loss = T.dissipation_mse(ke, dt, torch.tensor(eps_ref))
    loss.backward()
    return loss.item(), ke.detach().numpy(), th.grad.numpy()


def _dissipation_gpu(f0, theta, obs, dt, eps_ref, k):
    from paper_2412_08229_gb300.autograd import NCOKineticEnergyUnroll, dissipation_mse
    n = f0.shape[0]
    ctx = _ctx(n, "tgv_reduced", theta)
    th = torch.tensor(theta.astype(np.float32), device="cuda", requires_grad=True)
    f0d = torch.from_numpy(np.ascontiguousarray(np.moveaxis(f0, -1, 0)).astype(np.float32)).cuda()
    ke = NCOKineticEnergyUnroll.apply(th, ctx, f0d, obs, k)
    loss = dissipation_mse(ke, dt, torch.tensor(eps_ref, device="cuda"))
    loss.backward()
    return loss.item(), ke.detach().cpu().numpy(), th.grad.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("sizes", [DEEP, SHALLOW])
def test_dissipation_loss_gradient_reduced_domain(sizes):
    n, every, nsamp = 4, 2, 4
    obs = _obs(every, nsamp)
    dt = float(every)
    f0 = _start(n, "tgv_reduced")
    theta = _theta(sizes, seed=2)
    eps_ref = _eps_ref(f0, theta, obs, dt, sizes)
    l_ref, ke_ref, g_ref = _dissipation_reference(f0, theta, obs, dt, eps_ref, sizes)
    l_gpu, ke_gpu, g_gpu = _dissipation_gpu(f0, theta, obs, dt, eps_ref, k=3)
    assert np.abs(ke_gpu - ke_ref).max() <= 1e-6 * ke_ref.max()
    assert l_gpu == pytest.approx(l_ref, rel=1e-3)
    assert _rel(g_gpu, g_ref) <= 1e-3


@pytest.mark.parametrize("k", [1, 5, 20])
def test_kinetic_energy_gradient_does_not_depend_on_the_checkpoint_interval(k):
    n, every, nsamp = 4, 3, 3
    obs = _obs(every, nsamp)
    f0 = _start(n, "tgv_reduced")
    theta = _theta(DEEP, seed=2)
    eps_ref = _eps_ref(f0, theta, obs, float(every), DEEP)
    _, _, g2 = _dissipation_gpu(f0, theta, obs, float(every), eps_ref, k=2)
    _, _, gk = _dissipation_gpu(f0, theta, obs, float(every), eps_ref, k=k)
    assert _rel(gk, g2) <= 1e-6


def test_backward_ke_without_observations_equals_nco_backward():
    n = 4
    f0 = _start(n, "tgv_reduced")
    theta = _theta(DEEP)
    ctx = _ctx(n, "tgv_reduced", theta)
    G.set_gpu_state(ctx, np.moveaxis(f0, -1, 0))
    P.lbm_record_begin(ctx, 3)
    P.lbm_step(ctx, 5)
    u = torch.empty((3, n, n, n), device="cuda")
    P.lbm_macroscopic(ctx, None, u)
    a = torch.zeros(theta.size, device="cuda")
    b = torch.zeros(theta.size, device="cuda")
    P.nco_backward(ctx, u.contiguous(), None, a, None)
    P.nco_backward_ke(ctx, [], [], dL_du=u.contiguous(), dL_dtheta=b)
    assert _rel(b.cpu().numpy(), a.cpu().numpy()) <= 1e-6  # FP64 atomics may add in another order
    # the same observation given twice counts twice
    c = torch.zeros(theta.size, device="cuda")
    d = torch.zeros(theta.size, device="cuda")
    P.nco_backward_ke(ctx, [2], [2.0], dL_dtheta=c)
    P.nco_backward_ke(ctx, [2, 2], [1.0, 1.0], dL_dtheta=d)
    assert _rel(d.cpu().numpy(), c.cpu().numpy()) <= 1e-6


def test_backward_ke_refuses_bad_observations():
    n = 4
    theta = _theta(DEEP)
    ctx = _ctx(n, "tgv_reduced", theta)
    G.set_gpu_state(ctx, np.moveaxis(_start(n, "tgv_reduced"), -1, 0))
    P.lbm_record_begin(ctx, 2)
    P.lbm_step(ctx, 3)
    g = torch.zeros(theta.size, device="cuda")
    with pytest.raises(P.LbmError):
        P.nco_backward_ke(ctx, [4], [1.0], dL_dtheta=g)
    with pytest.raises(P.LbmError):
        P.nco_backward_ke(ctx, [-1], [1.0], dL_dtheta=g)
    with pytest.raises(P.LbmError):
        P.nco_backward_ke(ctx, [1], [float("nan")], dL_dtheta=g)
    with pytest.raises(P.LbmError):
        P.nco_backward_ke(ctx, [], [], dL_dtheta=g)
    assert P.lbm_check(ctx) == 0
