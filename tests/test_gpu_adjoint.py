"""GPU tests of nco_backward, the hand-written adjoint of the NCO step, against the FP64
references: autograd of the PyTorch restatement of the oracle, and central finite
differences (h = 1e-4, FP64) of the NumPy oracle.

Setting (the differentiation form at test size): Taylor-Green octant [0, pi]^3 on 8^3
nodes with mirror boundaries, 10 unrolled steps, loss = relative spectrum discrepancy
over shells 2..6 + 20 E(8) of the unfolded 16^3 field against a fixed reference spectrum.
Tolerance: 1e-3 relative (FP32 adjoint against FP64 references).
"""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from oracle import diagnostics as D
from oracle import stepper as S
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from oracle import torch_ref as T  # noqa: E402

N, STEPS, NU = 8, 10, 0.002
KMAX = N  # shells of the unfolded 2N box


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def _setup(n=N, bc="mirror"):
    if bc == "mirror":
        rho, u = lbm_inputs.taylor_green_octant(n, 0.05)
    else:
        rho, u = lbm_inputs.taylor_green_3d(n, 0.05)
    f0 = col.equilibrium(rho, np.moveaxis(u, 0, -1))          # (nz,ny,nx,27) float64
    f0 = f0.astype(np.float32).astype(np.float64)            # both sides start from FP32 values
    theta = lbm_inputs.nco_parameters(0).astype(np.float32).astype(np.float64)
    _, u0 = col.macroscopic(f0)
    uu = D.unfold_octant(u0) if bc == "mirror" else u0
    E_ref = 0.8 * D.energy_spectrum(uu, nbins=KMAX + 1) + 1e-10
    return f0, theta, E_ref


def _loss_torch(u_zyx3, E_ref, bc):
    uu = T.unfold_octant(u_zyx3) if bc == "mirror" else u_zyx3
    E = T.energy_spectrum(uu, KMAX + 1)
    return T.spectrum_loss(E, torch.tensor(E_ref), 2, KMAX - 2, 20.0, KMAX)


def _reference_grad(f0, theta, E_ref, nsteps, bc):
    th = torch.tensor(theta, requires_grad=True)
    f0t = torch.tensor(f0, requires_grad=True)
    f = T.run(f0t, col.tau_from_nu(NU), th, nsteps, bc=bc)
    loss = _loss_torch(T.velocity(f), E_ref, bc)
    loss.backward()
    return loss.item(), th.grad.numpy(), f0t.grad.numpy()


def _gpu_grad(f0, theta, E_ref, nsteps, bc, k):
    n = f0.shape[0]
    ctx = G.make_ctx((n, n, n), NU, "nco", bc=bc, theta=theta.astype(np.float32))
    G.set_gpu_state(ctx, np.moveaxis(f0, -1, 0))
    P.lbm_record_begin(ctx, k)
    P.lbm_step(ctx, nsteps)
    rho = torch.empty((n, n, n), device="cuda")
    u = torch.empty((3, n, n, n), device="cuda")
    P.lbm_macroscopic(ctx, rho, u)
    u64 = torch.tensor(np.moveaxis(u.cpu().numpy().astype(np.float64), 0, -1), requires_grad=True)
    loss = _loss_torch(u64, E_ref, bc)
    loss.backward()
    du = torch.from_numpy(np.ascontiguousarray(np.moveaxis(u64.grad.numpy(), -1, 0)).astype(np.float32)).cuda()
    dtheta = torch.zeros(1064, device="cuda")
    df0 = torch.zeros((27, n, n, n), device="cuda")
    P.nco_backward(ctx, du, None, dtheta, df0)
    torch.cuda.synchronize()
    return loss.item(), dtheta.cpu().numpy().astype(np.float64), np.moveaxis(df0.cpu().numpy(), 0, -1)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_adjoint_matches_autograd_reference_octant_8cube_10_steps():
    f0, theta, E_ref = _setup()
    l_ref, g_ref, gf_ref = _reference_grad(f0, theta, E_ref, STEPS, "mirror")
    l_gpu, g_gpu, gf_gpu = _gpu_grad(f0, theta, E_ref, STEPS, "mirror", k=3)
    assert l_gpu == pytest.approx(l_ref, rel=1e-3)
    assert _rel(g_gpu, g_ref) <= 1e-3
    assert _rel(gf_gpu, gf_ref) <= 1e-3


def test_adjoint_matches_central_differences_of_the_oracle():
    f0, theta, E_ref = _setup()
    _, g_gpu, _ = _gpu_grad(f0, theta, E_ref, STEPS, "mirror", k=4)

    def loss_np(th):
        f = S.Simulation(f0, col.tau_from_nu(NU), op="nco", theta=th, bc="mirror").step(STEPS).f
        _, u = col.macroscopic(f)
        E = D.energy_spectrum(D.unfold_octant(u), nbins=KMAX + 1)
        return D.spectrum_loss(E, E_ref, 2, KMAX - 2, 20.0, KMAX)

    h = 1e-4
    rng = np.random.default_rng(7)
    for _ in range(3):
        v = rng.standard_normal(theta.size)
        v /= np.linalg.norm(v)
        fd = (loss_np(theta + h * v) - loss_np(theta - h * v)) / (2 * h)
        assert g_gpu @ v == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.linalg.norm(g_gpu))


@pytest.mark.parametrize("k", [1, 4, 10])
def test_checkpoint_interval_does_not_change_the_gradient(k):
    f0, theta, E_ref = _setup(n=6)
    _, g3, _ = _gpu_grad(f0, theta, E_ref, 7, "mirror", k=3)
    _, gk, _ = _gpu_grad(f0, theta, E_ref, 7, "mirror", k=k)
    assert _rel(gk, g3) <= 1e-6


def test_adjoint_periodic_grid():
    f0, theta, E_ref = _setup(n=8, bc="periodic")
    l_ref, g_ref, gf_ref = _reference_grad(f0, theta, E_ref, 5, "periodic")
    l_gpu, g_gpu, gf_gpu = _gpu_grad(f0, theta, E_ref, 5, "periodic", k=2)
    assert _rel(g_gpu, g_ref) <= 1e-3
    assert _rel(gf_gpu, gf_ref) <= 1e-3


def test_autograd_function_returns_the_adjoint_gradient():
    from paper_2412_08229_gb300.autograd import NCOUnroll
    f0, theta, E_ref = _setup(n=6)
    ctx = G.make_ctx((6, 6, 6), NU, "nco", bc="mirror", theta=theta.astype(np.float32))
    th = torch.tensor(theta.astype(np.float32), device="cuda", requires_grad=True)
    f0d = torch.from_numpy(np.ascontiguousarray(np.moveaxis(f0, -1, 0)).astype(np.float32)).cuda()
    rho, u = NCOUnroll.apply(th, ctx, f0d, 7, 3)
    loss = (u.double() ** 2).sum() + (rho.double() ** 2).sum()
    loss.backward()
    _, g_ref, _ = _reference_grad_quadratic(f0, theta, 7)
    assert _rel(th.grad.cpu().numpy().astype(np.float64), g_ref) <= 1e-3


def _reference_grad_quadratic(f0, theta, nsteps):
    th = torch.tensor(theta, requires_grad=True)
    f = T.run(torch.tensor(f0), col.tau_from_nu(NU), th, nsteps, bc="mirror")
    loss = (T.velocity(f) ** 2).sum() + (f.sum(-1) ** 2).sum()
    loss.backward()
    return loss.item(), th.grad.numpy(), None


def _forced_reference_and_gpu(n, nsteps, power, k):
    """Forced turbulence on n^3 (periodic), nsteps recorded steps, loss sum |u|^2 + sum (rho-1)^2.
    The force of each step is an input of that step: the reference replays the force
    fields the oracle's own forward produced; the GPU replays the coefficients it recorded."""
    from oracle import forcing as F
    rho, u = lbm_inputs.isotropic_field(n, 1, 0.04)
    f0 = col.equilibrium(rho, np.moveaxis(u, 0, -1)).astype(np.float32).astype(np.float64)
    phi, psi = lbm_inputs.forcing_draws(nsteps, seed=3)
    theta = lbm_inputs.nco_parameters(0).astype(np.float32).astype(np.float64)
    tau = col.tau_from_nu(NU)
    rec = F.RecordedForcing(wrap=F.SpectralForcing(phi, psi, power=power))
    S.Simulation(f0, tau, op="nco", theta=theta, forcing=rec).step(nsteps)
    th = torch.tensor(theta, requires_grad=True)
    f0t = torch.tensor(f0, requires_grad=True)
    f = T.run(f0t, tau, th, nsteps, forces=rec.fields)
    loss = (T.velocity(f) ** 2).sum() + ((f.sum(-1) - 1.0) ** 2).sum()
    loss.backward()
    ctx = G.make_ctx((n, n, n), NU, "nco", theta=theta.astype(np.float32), forcing=dict(power=power))
    P.lbm_force_draws(ctx, phi, psi)
    G.set_gpu_state(ctx, np.moveaxis(f0, -1, 0))
    P.lbm_record_begin(ctx, k)
    P.lbm_step(ctx, nsteps)
    rho_d = torch.empty((n, n, n), device="cuda")
    u_d = torch.empty((3, n, n, n), device="cuda")
    P.lbm_macroscopic(ctx, rho_d, u_d)
    dtheta = torch.zeros(1064, device="cuda")
    df0 = torch.zeros((27, n, n, n), device="cuda")
    P.nco_backward(ctx, (2.0 * u_d).contiguous(), (2.0 * (rho_d - 1.0)).contiguous(), dtheta, df0)
    torch.cuda.synchronize()
    assert P.lbm_check(ctx) == 0
    return (th.grad.numpy(), f0t.grad.numpy(), dtheta.cpu().numpy().astype(np.float64),
            np.moveaxis(df0.cpu().numpy(), 0, -1).astype(np.float64))


def test_adjoint_through_forced_steps_matches_autograd_reference():
    g_ref, gf_ref, g_gpu, gf_gpu = _forced_reference_and_gpu(8, 6, 1e-5, k=4)
    assert _rel(g_gpu, g_ref) <= 1e-3
    assert _rel(gf_gpu, gf_ref) <= 1e-3


def _forced_reference_without_source_jacobian(n, nsteps, power):
    """The same reference gradient with the source term's dependence on f cut off."""
    from oracle import forcing as F
    rho, u = lbm_inputs.isotropic_field(n, 1, 0.04)
    f0 = col.equilibrium(rho, np.moveaxis(u, 0, -1)).astype(np.float32).astype(np.float64)
    phi, psi = lbm_inputs.forcing_draws(nsteps, seed=3)
    theta = lbm_inputs.nco_parameters(0).astype(np.float32).astype(np.float64)
    tau = col.tau_from_nu(NU)
    rec = F.RecordedForcing(wrap=F.SpectralForcing(phi, psi, power=power))
    S.Simulation(f0, tau, op="nco", theta=theta, forcing=rec).step(nsteps)
    th = torch.tensor(theta, requires_grad=True)
    f = torch.tensor(f0)
    for t in range(nsteps):
        fs = T.nco_collide(f, tau, th) + T.kupershtokh_source(f.detach(), torch.tensor(rec.fields[t]))
        f = T.stream_periodic(fs)
    loss = (T.velocity(f) ** 2).sum() + ((f.sum(-1) - 1.0) ** 2).sum()
    loss.backward()
    return th.grad.numpy()


def test_forced_adjoint_needs_the_source_jacobian_and_not_the_checkpoint_interval():
    """With a stronger force (power 1e-4: amplitude 0.028 per step against u_rms 0.04) the
    source's Jacobian moves the gradient by 0.9 %, several times the tolerance, so the match
    shows the adjoint includes it; the checkpoint interval does not change the gradient."""
    g_ref, _, g_gpu, _ = _forced_reference_and_gpu(8, 5, 1e-4, k=1)
    _, _, g_gpu5, _ = _forced_reference_and_gpu(8, 5, 1e-4, k=5)
    g_cut = _forced_reference_without_source_jacobian(8, 5, 1e-4)
    assert _rel(g_cut, g_ref) > 5e-3
    assert _rel(g_gpu, g_ref) <= 1e-3
    assert _rel(g_gpu5, g_gpu) <= 1e-6


def test_kinetic_energy_observations_through_forced_steps():
    """nco_backward_ke on a forced context: loss = sum of k after 0, 3 and 6 steps, the
    force of each step an input (the reference replays the oracle's force fields)."""
    from oracle import forcing as F
    n, nsteps, power = 8, 6, 1e-5
    obs = [0, 3, 6]
    rho, u = lbm_inputs.isotropic_field(n, 1, 0.04)
    f0 = col.equilibrium(rho, np.moveaxis(u, 0, -1)).astype(np.float32).astype(np.float64)
    phi, psi = lbm_inputs.forcing_draws(nsteps, seed=3)
    theta = lbm_inputs.nco_parameters(0).astype(np.float32).astype(np.float64)
    tau = col.tau_from_nu(NU)
    rec = F.RecordedForcing(wrap=F.SpectralForcing(phi, psi, power=power))
    S.Simulation(f0, tau, op="nco", theta=theta, forcing=rec).step(nsteps)
    th = torch.tensor(theta, requires_grad=True)
    f, loss = torch.tensor(f0), 0.0
    for t in range(nsteps + 1):
        if t in obs:
            loss = loss + T.kinetic_energy(f)
        if t < nsteps:
            f = T.stream_periodic(T.nco_collide(f, tau, th) + T.kupershtokh_source(f, torch.tensor(rec.fields[t])))
    loss.backward()
    ctx = G.make_ctx((n, n, n), NU, "nco", theta=theta.astype(np.float32), forcing=dict(power=power))
    P.lbm_force_draws(ctx, phi, psi)
    G.set_gpu_state(ctx, np.moveaxis(f0, -1, 0))
    P.lbm_record_begin(ctx, 4)
    P.lbm_step(ctx, nsteps)
    g = torch.zeros(1064, device="cuda")
    P.nco_backward_ke(ctx, obs, [1.0, 1.0, 1.0], dL_dtheta=g)
    torch.cuda.synchronize()
    assert _rel(g.cpu().numpy().astype(np.float64), th.grad.numpy()) <= 1e-3
