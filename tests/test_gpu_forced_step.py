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
