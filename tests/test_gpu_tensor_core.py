"""GPU tests of the tcgen05 (BF16 operand, FP32 accumulate) network form of the NCO step.

One-step parity: the reference is the FP64 oracle with the network's operands rounded to
BF16 as the kernel rounds them, and every stored population must be a storage rounding of
a value within the bound of tests/bf16_ref.py (rounding ambiguities of the BF16 inputs and
activations to first order in the network's Jacobian, FP32 arithmetic). Each case runs
with the seed-0 Kaiming weights and with state-sensitive weights (W1 x 30), on random
populations far from equilibrium; tests/test_bf16_tolerance.py shows on the CPU that the
check rejects a constant-rate network, a missing or wrong group action and a wrong input
layout on these inputs. Multi-step and kinetic-energy tests compare with the plain oracle.
"""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from oracle import diagnostics as D
from oracle import lattice as L
from oracle import stepper as S
from tests import bf16_ref as B
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

WEIGHTS = ("seed0", "sensitive")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.P._abi.load()


def test_tcgen05_gemm_selftest_is_exact():
    assert P.lbm_selftest_tensor_cores() == 0.0


@pytest.mark.parametrize("weights", WEIGHTS)
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("bc", B.CASES["ragged"][4])
def test_bf16_network_one_step_ragged(storage, bc, weights):
    """Random populations on 7x6x5 (ragged last tile of 128 cells: 210 = 128 + 82)."""
    shape, seed, nu, sizes, _ = B.CASES["ragged"]
    theta = B.case_theta(sizes, weights)
    ctx = G.make_ctx(shape, nu, "nco", storage=storage, net="bf16", bc=bc, theta=theta)
    G.set_gpu_state(ctx, lbm_inputs.random_populations(shape, seed))
    G.check_bf16_step(ctx, nu, theta, sizes, bc, storage)


@pytest.mark.parametrize("weights", WEIGHTS)
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_bf16_network_large_ragged_grid(storage, weights):
    """A grid spanning 40 tiles over several warpgroups and SMs with a ragged tail (33x17x9 = 5049 cells)."""
    shape, seed, nu, sizes, _ = B.CASES["large_ragged"]
    theta = B.case_theta(sizes, weights)
    ctx = G.make_ctx(shape, nu, "nco", storage=storage, net="bf16", theta=theta)
    G.set_gpu_state(ctx, lbm_inputs.random_populations(shape, seed))
    G.check_bf16_step(ctx, nu, theta, sizes, "periodic", storage)


def test_bf16_network_with_several_tiles_per_pipeline():
    """48 x 40 x 32 = 61,440 cells = 480 tiles, more than the 2 x 152 tile pipelines of the
    pair kernel, so pipelines step from one tile to the next (the hand-over of the shared
    layer-1 operand and of the group sums between the two warpgroups): every population
    of one step meets the BF16 oracle bound (random populations, mixed form)."""
    shape, nu = (32, 40, 48), 0.01
    theta = G.theta0()
    ctx = G.make_ctx(shape, nu, "nco", storage="f16", net="bf16", theta=theta)
    G.set_gpu_state(ctx, lbm_inputs.random_populations(shape, 23))
    G.check_bf16_step(ctx, nu, theta, storage="f16")


@pytest.mark.parametrize("storage,net,deep", [("f16", "bf16", False), ("f32", "bf16", False),
                                               ("f16", "bf16", True), ("f32", "bf16x3", False)],
                         ids=["pair-f16", "pair-f32", "chunked-deep-f16", "split-f32"])
def test_tensor_core_runs_are_bit_reproducible_over_many_tile_handovers(storage, net, deep):
    """64^3 = 2048 tiles, about 7 per tile pipeline of the pair kernel, over 1000 steps:
    about 1.7 M hand-overs of the shared layer-1 operand and of the group sums between the
    two warpgroups of a pipeline. Two runs end in the same state bit for bit. A hand-over
    that let one warpgroup overwrite the operand while the other's last layer-1 MMA of the
    tile was still pending would make the runs differ (the result would depend on timing).
    The chunked kernel (deep network) and the split-BF16 kernel, whose warpgroups wait only
    on their own commits, are held to the same."""
    n, nu = 64, 0.002
    rho, u = lbm_inputs.taylor_green_3d(n, 0.05)
    theta = B.case_theta(B.DEEP_SIZES, "seed0") if deep else G.theta0()

    def run():
        ctx = G.make_ctx((n, n, n), nu, "nco", storage=storage, net=net, theta=theta)
        G.init_gpu(ctx, rho, u)
        P.lbm_step(ctx, 1000)
        assert P.lbm_check(ctx) == 0
        raw = P.lbm_get_raw_state(ctx)
        P.lbm_destroy(ctx)
        return raw

    assert np.array_equal(run(), run())


def test_bf16_network_on_tgv16_step_by_step():
    """Config 0 geometry: the FP32 network meets 1e-5 after 3 steps; the BF16 one meets
    the BF16 bound at each of 3 steps, each checked from the state the GPU reached."""
    rho, u = lbm_inputs.taylor_green_3d(16, 0.05)
    nu = 0.005
    theta = G.theta0()
    a = G.make_ctx((16,) * 3, nu, "nco", net="f32", theta=theta)
    b = G.make_ctx((16,) * 3, nu, "nco", net="bf16", theta=theta)
    for c in (a, b):
        G.init_gpu(c, rho, u)
    P.lbm_step(a, 3)
    sim = G.oracle_sim_from_fields(rho, u, col.tau_from_nu(nu), "nco", theta=theta)
    assert G.rel_maxnorm(G.to_oracle_f(G.gpu_state(a)), sim.step(3).f) <= 1e-5
    for _ in range(3):
        G.check_bf16_step(b, nu, theta)


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
    sim.operand_round = B.bf16
    th = theta.astype(np.float64)
    budget = 0.0
    for _ in range(3):  # the BF16 bound of every step the oracle takes, plus FP32 arithmetic
        budget += (B.population_bound(sim.f, B.rate_bound(sim.f, th)).max() + 1e-5 * np.abs(sim.f).max())
        sim.step(1)
    assert np.abs(got - sim.f).max() <= budget
