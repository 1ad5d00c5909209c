"""GPU tests of the tcgen05 (BF16 operand, FP32 accumulate) network form of the NCO step.

Tolerance of the BF16 network: every learned rate omega_n = 1/tau_n may move by at
most 1e-2 (inputs and weights carry 8 significant bits, d omega / d tau~ <= 1/2, and the
mean over 48 elements averages the rounding), so the populations may move by at most
1e-2 * max|M^-1 m_{>=3}|, the size of the higher-order non-equilibrium part the rates
act on; storage rounding and the FP32 allowance come on top.
"""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from oracle import diagnostics as D
from oracle import lattice as L
from oracle import stepper as S
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

HALF_ULP = {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}
RATE_TOL = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.P._abi.load()


def test_tcgen05_gemm_selftest_is_exact():
    assert P.lbm_selftest_tensor_cores() == 0.0


def _higher_order_part(f):
    """max over cells of |M^-1 (m_{>=3})|, the part of f the learned rates relax."""
    m = col.moments(f)
    mh = np.where(L.MOMENT_ORDER >= 3, m, 0.0)
    return float(np.abs(mh @ L.M_INV.T).max())


def _tol(start, ref, storage):
    return (RATE_TOL * _higher_order_part(start) + HALF_ULP[storage] * np.abs(ref - L.W).max()
            + 1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("bc", ["periodic", "mirror"])
def test_bf16_network_one_step_ragged(storage, bc):
    """Random populations on 7x6x5 (ragged last tile of 128 cells: 210 = 128 + 82)."""
    shape = (7, 6, 5)
    f0 = lbm_inputs.random_populations(shape, 17)
    nu = 0.02
    theta = G.theta0()
    ctx = G.make_ctx(shape, nu, "nco", storage=storage, net="bf16", bc=bc, theta=theta)
    G.set_gpu_state(ctx, f0)
    start = G.to_oracle_f(G.gpu_state(ctx))
    P.lbm_step(ctx, 1)
    assert P.lbm_check(ctx) == 0
    got = G.to_oracle_f(G.gpu_state(ctx))
    sim = S.Simulation(start, col.tau_from_nu(nu), op="nco", theta=theta.astype(np.float64), bc=bc)
    ref = sim.step(1).f
    assert np.abs(got - ref).max() <= _tol(start, ref, storage)


def _oracle_steps_with_budget(sim, nsteps):
    """Advance the oracle and sum the rate-tolerance budget of every step it takes."""
    budget = 0.0
    for _ in range(nsteps):
        budget += RATE_TOL * _higher_order_part(sim.f)
        sim.step(1)
    return sim.f, budget


def test_bf16_network_matches_fp32_network_on_tgv16():
    """Config 0 geometry: the FP32 network meets 1e-5, the BF16 one the rate tolerance."""
    rho, u = lbm_inputs.taylor_green_3d(16, 0.05)
    nu = 0.005
    theta = G.theta0()
    a = G.make_ctx((16,) * 3, nu, "nco", net="f32", theta=theta)
    b = G.make_ctx((16,) * 3, nu, "nco", net="bf16", theta=theta)
    for c in (a, b):
        G.init_gpu(c, rho, u)
    P.lbm_step(a, 3)
    P.lbm_step(b, 3)
    fa, fb = G.to_oracle_f(G.gpu_state(a)), G.to_oracle_f(G.gpu_state(b))
    sim = G.oracle_sim_from_fields(rho, u, col.tau_from_nu(nu), "nco", theta=theta)
    ref, budget = _oracle_steps_with_budget(sim, 3)
    assert G.rel_maxnorm(fa, ref) <= 1e-5
    assert np.abs(fb - ref).max() <= budget + 1e-5 * np.abs(ref).max()


def test_bf16_network_equivariance_all_48():
    f0 = lbm_inputs.random_populations((4, 4, 4), 29)
    theta = G.theta0()
    ctx = G.make_ctx((4, 4, 4), 0.02, "nco", net="bf16", theta=theta)
    G.set_gpu_state(ctx, f0)
    P.lbm_step(ctx, 1)
    from tests.test_gpu_parity import _transform_soa
    base = G.gpu_state(ctx)
    for g in range(48):
        G.set_gpu_state(ctx, _transform_soa(f0, g))
        P.lbm_step(ctx, 1)
        assert np.abs(G.gpu_state(ctx) - _transform_soa(base, g)).max() <= 1e-6, g


def test_mixed_form_kinetic_energy_curve_16cube():
    """FP16 deviation storage + BF16 network: KE within 1e-3 of the FP64 oracle over 1000 steps."""
    rho, u = lbm_inputs.taylor_green_3d(16, 0.05)
    nu = 0.005
    theta = G.theta0()
    ctx = G.make_ctx((16,) * 3, nu, "nco", storage="f16", net="bf16", theta=theta)
    G.init_gpu(ctx, rho, u)
    sim = G.oracle_sim_from_fields(rho, u, col.tau_from_nu(nu), "nco", theta=theta)
    worst = 0.0
    for _ in range(10):
        P.lbm_step(ctx, 100)
        sim.step(100)
        ke = P.lbm_kinetic_energy(ctx)
        ref = D.kinetic_energy(sim.macroscopic()[1])
        worst = max(worst, abs(ke - ref) / ref)
    assert P.lbm_check(ctx) == 0
    assert worst <= 1e-3, worst


def test_bf16_network_large_ragged_grid():
    """A grid spanning many tiles and both warpgroups with a ragged tail (33x17x9 = 5049 cells)."""
    shape = (9, 17, 33)
    rng = np.random.default_rng(4)
    u = rng.standard_normal((3,) + shape) * 0.03
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    nu = 0.01
    theta = G.theta0()
    ctx = G.make_ctx(shape, nu, "nco", storage="f32", net="bf16", theta=theta)
    G.init_gpu(ctx, rho, u)
    P.lbm_step(ctx, 2)
    got = G.to_oracle_f(G.gpu_state(ctx))
    sim = G.oracle_sim_from_fields(rho, u, col.tau_from_nu(nu), "nco", theta=theta)
    ref, budget = _oracle_steps_with_budget(sim, 2)
    assert np.abs(got - ref).max() <= budget + 1e-5 * np.abs(ref).max()


def test_bf16_network_forced():
    from oracle import forcing as F
    n = 16
    rho, u = lbm_inputs.isotropic_field(n, 1, 0.04)
    nu, power = 0.0015, 1e-6
    phi, psi = lbm_inputs.forcing_draws(3, seed=3)
    theta = G.theta0()
    ctx = G.make_ctx((n, n, n), nu, "nco", net="bf16", theta=theta, forcing=dict(power=power))
    G.init_gpu(ctx, rho, u)
    P.lbm_force_draws(ctx, phi, psi)
    P.lbm_step(ctx, 3)
    got = G.to_oracle_f(G.gpu_state(ctx))
    forcing = F.SpectralForcing(phi, psi, power=power)
    sim = G.oracle_sim_from_fields(rho, u, col.tau_from_nu(nu), "nco", theta=theta, forcing=forcing)
    ref, budget = _oracle_steps_with_budget(sim, 3)
    assert np.abs(got - ref).max() <= budget + 1e-5 * np.abs(ref).max()
