"""Pins of the differentiable FP64 restatement (oracle.torch_ref), CPU only.

Its forward equals the NumPy oracle's, and its autograd gradient of the spectrum loss
through an unrolled NCO simulation equals central finite differences of the NumPy oracle.
"""

import numpy as np
import pytest

import lbm_inputs
from oracle import collision as col
from oracle import diagnostics as D
from oracle import stepper as S

torch = pytest.importorskip("torch")
from oracle import torch_ref as T  # noqa: E402


def _octant(n, u0=0.05):
    rho, u = lbm_inputs.taylor_green_octant(n, u0)
    return col.equilibrium(rho, np.moveaxis(u, 0, -1))


@pytest.mark.parametrize("bc", ["periodic", "mirror"])
def test_torch_restatement_forward_equals_numpy_oracle(bc):
    f0 = np.moveaxis(lbm_inputs.random_populations((3, 4, 5), 61), 0, -1)
    theta = lbm_inputs.nco_parameters(0)
    tau = 0.58
    ref = S.Simulation(f0, tau, op="nco", theta=theta, bc=bc).step(3).f
    got = T.run(torch.tensor(f0), tau, torch.tensor(theta), 3, bc=bc).numpy()
    assert np.allclose(got, ref, atol=1e-14)


def _loss_numpy(theta, f0, tau, nsteps, E_ref, kmax):
    f = S.Simulation(f0, tau, op="nco", theta=theta, bc="mirror").step(nsteps).f
    _, u = col.macroscopic(f)
    E = D.energy_spectrum(D.unfold_octant(u), nbins=kmax + 1)
    return D.spectrum_loss(E, E_ref, 2, kmax, 20.0, kmax)


def test_autograd_gradient_matches_central_differences_of_the_oracle():
    n, nsteps, tau = 4, 3, 0.52
    f0 = _octant(n)
    theta = lbm_inputs.nco_parameters(0)
    kmax = n  # full box 2n: shells up to n
    _, u_init = col.macroscopic(f0)
    E_ref = 0.9 * D.energy_spectrum(D.unfold_octant(u_init), nbins=kmax + 1) + 1e-12
    th = torch.tensor(theta, requires_grad=True)
    f = T.run(torch.tensor(f0), tau, th, nsteps, bc="mirror")
    E = T.energy_spectrum(T.unfold_octant(T.velocity(f)), kmax + 1)
    loss = T.spectrum_loss(E, torch.tensor(E_ref), 2, kmax, 20.0, kmax)
    loss.backward()
    grad = th.grad.numpy()
    assert loss.item() == pytest.approx(_loss_numpy(theta, f0, tau, nsteps, E_ref, kmax), rel=1e-12)
    h = 1e-4
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.standard_normal(theta.size)
        v /= np.linalg.norm(v)
        fd = (_loss_numpy(theta + h * v, f0, tau, nsteps, E_ref, kmax)
              - _loss_numpy(theta - h * v, f0, tau, nsteps, E_ref, kmax)) / (2 * h)
        assert grad @ v == pytest.approx(fd, rel=1e-6, abs=1e-12)
    for k in rng.choice(theta.size, size=6, replace=False):
        e = np.zeros(theta.size)
        e[k] = 1.0
        fd = (_loss_numpy(theta + h * e, f0, tau, nsteps, E_ref, kmax)
              - _loss_numpy(theta - h * e, f0, tau, nsteps, E_ref, kmax)) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def _forced_setup(n=6, nsteps=4, power=1e-5):
    from oracle import forcing as F
    rho, u = lbm_inputs.isotropic_field(n, 1, 0.04)
    f0 = col.equilibrium(rho, np.moveaxis(u, 0, -1))
    phi, psi = lbm_inputs.forcing_draws(nsteps, seed=3)
    rec = F.RecordedForcing(wrap=F.SpectralForcing(phi, psi, power=power))
    theta = lbm_inputs.nco_parameters(0)
    tau = 0.53
    ref = S.Simulation(f0, tau, op="nco", theta=theta, forcing=rec).step(nsteps).f
    return f0, theta, tau, rec.fields, ref


def test_torch_restatement_with_forces_equals_the_forced_oracle():
    f0, theta, tau, fields, ref = _forced_setup()
    got = T.run(torch.tensor(f0), tau, torch.tensor(theta), len(fields), forces=fields).numpy()
    assert np.abs(got - ref).max() <= 1e-14
    # the forces act: without them the state differs by far more than rounding
    plain = T.run(torch.tensor(f0), tau, torch.tensor(theta), len(fields)).numpy()
    assert np.abs(plain - ref).max() > 1e-9


def test_autograd_gradient_through_forced_steps_matches_central_differences():
    """The force fields are inputs of the steps (the oracle replays the recorded fields)."""
    from oracle import forcing as F
    f0, theta, tau, fields, _ = _forced_setup()
    nsteps = len(fields)

    def loss_np(th):
        f = S.Simulation(f0, tau, op="nco", theta=th, forcing=F.RecordedForcing(fields)).step(nsteps).f
        rho, u = col.macroscopic(f)
        return float((u * u).sum() + ((rho - 1.0) ** 2).sum())

    th = torch.tensor(theta, requires_grad=True)
    f = T.run(torch.tensor(f0), tau, th, nsteps, forces=fields)
    loss = (T.velocity(f) ** 2).sum() + ((f.sum(-1) - 1.0) ** 2).sum()
    loss.backward()
    g = th.grad.numpy()
    assert loss.item() == pytest.approx(loss_np(theta), rel=1e-12)
    # h = 1e-5: a ReLU kink close along a direction makes the difference quotient converge
    # only as fast as h shrinks (measured: 5e-5, 1.5e-5, 3.6e-6 relative at h = 1e-3..1e-5),
    # hence the absolute allowance of 1e-7 of the gradient's norm
    h = 1e-5
    rng = np.random.default_rng(9)
    for _ in range(3):
        v = rng.standard_normal(theta.size)
        v /= np.linalg.norm(v)
        fd = (loss_np(theta + h * v) - loss_np(theta - h * v)) / (2 * h)
        assert g @ v == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.linalg.norm(g))
