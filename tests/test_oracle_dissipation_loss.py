"""CPU pins of the dissipation loss of Sec. IV (training on time-dependent data) and of the
PyTorch restatement's reduced-domain, deep-network and kinetic-energy parts.

The loss is the mean squared difference between -dk/dt and a reference at 100 points
between t = 0 and t = 15; -dk/dt comes from central differences of k sampled on a uniform
grid (oracle.diagnostics). Pins: the exact central difference of an exponential, the
sampling grid, and central finite differences of the NumPy oracle for the gradient that
autograd of the restatement gives through an unrolled reduced-domain simulation.
"""

import math

import numpy as np
import pytest

import lbm_inputs
from oracle import collision as col
from oracle import diagnostics as D
from oracle import stepper as S

torch = pytest.importorskip("torch")
from oracle import torch_ref as T  # noqa: E402

DEEP = (27, 20, 20, 20, 4)


def test_sampling_grid_has_100_interior_points_in_0_15():
    t, dt = D.dissipation_sample_times()
    assert t.size == 102 and t[0] == 0.0 and t[-1] == pytest.approx(15.0, rel=1e-15)
    assert np.allclose(np.diff(t), dt, rtol=1e-12)
    inner = t[1:-1]
    assert inner.size == D.DISSIPATION_SAMPLES == 100
    assert inner.min() > 0.0 and inner.max() < 15.0


def test_loss_of_an_exponential_decay_against_its_exact_derivative():
    # k = a exp(-b t): the central difference is a exp(-b t) sinh(b dt) / dt exactly,
    # the exact dissipation a b exp(-b t)
    a, b = 0.3, 0.4
    t, dt = D.dissipation_sample_times()
    ke = a * np.exp(-b * t)
    inner = t[1:-1]
    eps_exact = a * b * np.exp(-b * inner)
    got = D.dissipation_mse(ke, dt, eps_exact)
    want = np.mean((a * np.exp(-b * inner)) ** 2) * (math.sinh(b * dt) / dt - b) ** 2
    assert got == pytest.approx(want, rel=1e-9)
    assert got > 0.0


def test_loss_is_zero_against_its_own_curve_and_quadratic_in_the_offset():
    t, dt = D.dissipation_sample_times(t_end=3.0, nsamples=7)
    ke = 1.0 / (1.0 + t) + 0.01 * np.sin(5 * t)
    eps = D.dissipation(ke, dt)
    assert D.dissipation_mse(ke, dt, eps) == 0.0
    assert D.dissipation_mse(ke, dt, eps + 0.25) == pytest.approx(0.0625, rel=1e-12)
    # k rising in time is negative dissipation
    assert (D.dissipation(t, dt) == pytest.approx(-1.0))


def test_loss_rejects_a_reference_of_the_wrong_length():
    with pytest.raises(ValueError):
        D.dissipation_mse(np.ones(10), 0.1, np.ones(9))


def test_torch_restatement_of_the_loss_equals_the_oracle():
    t, dt = D.dissipation_sample_times(t_end=2.0, nsamples=9)
    rng = np.random.default_rng(5)
    ke = np.exp(-t) + 0.001 * rng.standard_normal(t.size)
    ref = rng.uniform(0.5, 1.0, 9)
    assert T.dissipation_mse(torch.tensor(ke), dt, torch.tensor(ref)).item() == pytest.approx(
        D.dissipation_mse(ke, dt, ref), rel=1e-13)


def _reduced_start(n, u0=0.05):
    rho, u = lbm_inputs.taylor_green_3d(4 * n, u0, shifted=True)
    return col.equilibrium(rho[:n, :n, :n], np.moveaxis(u[:, :n, :n, :n], 0, -1))


def test_torch_restatement_reduced_domain_deep_network_equals_the_oracle():
    n, tau = 3, 0.55
    f0 = _reduced_start(n)
    theta = lbm_inputs.nco_parameters(1, DEEP)
    ref = S.Simulation(f0, tau, op="nco", theta=theta, bc="tgv_reduced", sizes=DEEP).step(3).f
    got = T.run(torch.tensor(f0), tau, torch.tensor(theta), 3, bc="tgv_reduced", sizes=DEEP).numpy()
    assert np.abs(got - ref).max() <= 1e-14


def _oracle_ke_curve(theta, f0, tau, obs, sizes):
    sim = S.Simulation(f0, tau, op="nco", theta=theta, bc="tgv_reduced", sizes=sizes)
    out, t = [], 0
    for s in obs:
        sim.step(s - t)
        t = s
        _, u = col.macroscopic(sim.f)
        out.append(D.kinetic_energy(u))
    return np.array(out)


def test_autograd_dissipation_loss_gradient_matches_central_differences_of_the_oracle():
    n, tau, every, nsamp = 2, 0.52, 2, 3
    obs = [every * j for j in range(nsamp + 2)]
    dt = float(every)
    f0 = _reduced_start(n)
    theta = lbm_inputs.nco_parameters(0, DEEP)
    eps_ref = 0.5 * D.dissipation(_oracle_ke_curve(theta, f0, tau, obs, DEEP), dt)

    th = torch.tensor(theta, requires_grad=True)
    ke = T.run_kinetic_energy(torch.tensor(f0), tau, th, obs, bc="tgv_reduced", sizes=DEEP)
    loss = T.dissipation_mse(ke, dt, torch.tensor(eps_ref))
    loss.backward()
    g = th.grad.numpy()

    def loss_np(t_):
        return D.dissipation_mse(_oracle_ke_curve(t_, f0, tau, obs, DEEP), dt, eps_ref)

    assert loss.item() == pytest.approx(loss_np(theta), rel=1e-12)
    h = 1e-4
    rng = np.random.default_rng(11)
    for _ in range(2):
        v = rng.standard_normal(theta.size)
        v /= np.linalg.norm(v)
        fd = (loss_np(theta + h * v) - loss_np(theta - h * v)) / (2 * h)
        assert g @ v == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.linalg.norm(g))
