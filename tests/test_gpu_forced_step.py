"""The forced step's in-kernel projection (Sec. II.C) is summed in fixed point, so its
result does not depend on the order in which warps add to it: a forced run is bit-for-bit
reproducible, and the CUDA-graph replay of lbm_step(ctx, n) equals the same steps
launched one at a time. Checked on a grid whose warps span two rows (ragged last tile)
and on one whose warps lie within a row, for the CUDA-core operators and both
tensor-core network forms."""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

STEPS = 12
FORMS = [("bgk", "f32", "f32"), ("kbc", "f32", "f32"), ("nco", "f32", "f32"), ("nco", "f16", "bf16"),
         ("nco", "f32", "bf16x3")]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def _run(shape, op, storage, net, one_at_a_time):
    ctx = G.make_ctx(shape, 0.002, op, storage=storage, net=net, theta=G.theta0(), forcing=dict(power=2e-6))
    rng = np.random.default_rng(7)
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.03 * rng.standard_normal((3,) + shape)
    G.init_gpu(ctx, rho, u)
    phi, psi = lbm_inputs.forcing_draws(STEPS, seed=11)
    P.lbm_force_draws(ctx, phi, psi)
    if one_at_a_time:
        for _ in range(STEPS):
            P.lbm_step(ctx, 1)
    else:
        P.lbm_step(ctx, STEPS)
    assert P.lbm_check(ctx) == 0
    f = G.gpu_state(ctx)
    P.lbm_destroy(ctx)
    return f


@pytest.mark.parametrize("shape", [(18, 20, 24), (16, 8, 32)])
@pytest.mark.parametrize("form", FORMS, ids=lambda f: "-".join(f))
def test_forced_runs_are_bit_reproducible_and_graph_replay_equals_direct_steps(shape, form):
    a = _run(shape, *form, one_at_a_time=False)
    b = _run(shape, *form, one_at_a_time=False)
    c = _run(shape, *form, one_at_a_time=True)
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)


@pytest.mark.parametrize("form", [("bgk", "f32", "f32"), ("nco", "f16", "bf16"), ("nco", "f32", "f32")],
                         ids=lambda f: "-".join(f))
def test_forced_run_resumes_bit_for_bit_from_raw_and_force_state(form):
    """Checkpoint/resume: a forced run saved after 6 of 12 steps (lbm_get_raw_state's stored
    state and lbm_get_force_state's projection sums) and restored into a fresh context, with
    the remaining draws queued, ends in the same state bit for bit as the uninterrupted run.
    Without the force state the resumed run differs (the restored context projects the
    restored state, not the velocity of the step before it)."""
    shape = (16, 12, 20)
    full = _run(shape, *form, one_at_a_time=False)
    op, storage, net = form
    phi, psi = lbm_inputs.forcing_draws(STEPS, seed=11)
    rng = np.random.default_rng(7)
    rho = 1.0 + 0.01 * rng.standard_normal(shape)
    u = 0.03 * rng.standard_normal((3,) + shape)
    half = STEPS // 2
    a = G.make_ctx(shape, 0.002, op, storage=storage, net=net, theta=G.theta0(), forcing=dict(power=2e-6))
    G.init_gpu(a, rho, u)
    P.lbm_force_draws(a, phi[:half], psi[:half])
    P.lbm_step(a, half)
    raw = P.lbm_get_raw_state(a)
    sums = P.lbm_get_force_state(a)
    P.lbm_destroy(a)

    def resume(with_force_state):
        b = G.make_ctx(shape, 0.002, op, storage=storage, net=net, theta=G.theta0(), forcing=dict(power=2e-6))
        P.lbm_set_raw_state(b, raw)
        if with_force_state:
            P.lbm_set_force_state(b, sums)
        P.lbm_force_draws(b, phi[half:], psi[half:])
        P.lbm_step(b, STEPS - half)
        assert P.lbm_check(b) == 0
        f = G.gpu_state(b)
        P.lbm_destroy(b)
        return f

    assert np.array_equal(resume(True), full)
    assert not np.array_equal(resume(False), full)
