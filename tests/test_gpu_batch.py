"""GPU tests of the batched form: independent NCO instances of uneven size stepped by one
persistent tensor-core launch per step, directly or replayed from CUDA graphs.

Each instance of a batch must evolve exactly as the same instance stepped on its own
with lbm_step (the batched kernel runs the same per-cell arithmetic), whatever the mode,
the chunking of the steps, the autotuned launch shape, or direct steps of one instance
between replays.
"""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

POWER = 2e-6
SPECS = [  # (nz, ny, nx), nu, forced, field
    ((16, 16, 16), 0.004, False, "tgv"),
    ((18, 20, 24), 0.002, False, "random"),   # 8640 cells: a ragged last tile
    ((16, 16, 16), 0.003, True, "hit"),
    ((8, 8, 8), 0.01, False, "random"),
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def _fields(shape, kind, seed):
    nz, ny, nx = shape
    if kind == "tgv":
        return lbm_inputs.taylor_green_3d(nx, 0.05)
    if kind == "hit":
        return lbm_inputs.isotropic_field(nx, seed=1, u_rms=0.04)
    rng = np.random.default_rng(seed)
    return 1.0 + 0.01 * rng.standard_normal(shape), 0.03 * rng.standard_normal((3,) + shape)


def _spec_kwargs(shape, nu, forced, storage):
    nz, ny, nx = shape
    return dict(nx=nx, ny=ny, nz=nz, nu=nu, storage=storage, forcing=dict(power=POWER) if forced else None)


def _draws(steps):
    return lbm_inputs.forcing_draws(steps, seed=5)


def _setup_instance(ctx, i, steps):
    shape, _, forced, kind = SPECS[i]
    rho, u = _fields(shape, kind, 10 + i)
    G.init_gpu(ctx, rho, u)
    if forced:
        phi, psi = _draws(steps)
        P.lbm_force_draws(ctx, phi, psi)


def _batch(storage, steps):
    b = P.lbm_batch_create([_spec_kwargs(s, nu, fo, storage) for s, nu, fo, _ in SPECS])
    P.lbm_batch_set_weights(b, G.theta0())
    for i in range(len(SPECS)):
        _setup_instance(b[i], i, steps)
    return b


def _individual(i, storage, steps, nsteps):
    shape, nu, forced, _ = SPECS[i]
    ctx = G.make_ctx(shape, nu, "nco", storage=storage, net="bf16", theta=G.theta0(),
                     forcing=dict(power=POWER) if forced else None)
    _setup_instance(ctx, i, steps)
    P.lbm_step(ctx, nsteps)
    return G.gpu_state(ctx)


def _states(b):
    torch.cuda.synchronize()
    return [G.gpu_state(b[i]) for i in range(len(SPECS))]


@pytest.mark.parametrize("storage", ["f16", "f32"])
@pytest.mark.parametrize("modes", [(True, True), (False, False), (False, True)])
def test_batch_equals_instances_stepped_alone(storage, modes):
    steps = 7
    b = _batch(storage, steps)
    for chunk, use_graph in zip((3, 4), modes):  # calls continue each other (odd chunk: the other parity next)
        P.lbm_batch_step(b, chunk, use_graph=use_graph)
    assert P.lbm_batch_check(b) == 0
    got = _states(b)
    for i in range(len(SPECS)):
        ref = _individual(i, storage, steps, steps)
        assert np.array_equal(got[i], ref), f"instance {i}"


def test_graph_and_direct_modes_agree_and_autotune_keeps_the_state():
    steps = 6
    a, b = _batch("f16", steps), _batch("f16", steps)
    before = _states(b)
    choice = P.lbm_batch_autotune(b)
    assert choice in (0, 2, 3, 4)
    after = _states(b)
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    P.lbm_batch_set_tile_shape(a, choice)
    P.lbm_batch_step(a, steps, use_graph=False)
    P.lbm_batch_step(b, steps, use_graph=True)
    for x, y in zip(_states(a), _states(b)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("shape", [0, 2, 4])
def test_every_tile_shape_follows_its_instances_stepped_alone(shape):
    """In each tile shape a batch instance stepped alone with lbm_step (which then uses the
    batch's shape) follows the batch bit for bit; the shapes agree with each other within the
    BF16 network's accuracy (they differ in the rounding order of FP32 sums)."""
    steps = 4
    b = _batch("f16", steps)
    P.lbm_batch_set_tile_shape(b, shape)
    P.lbm_batch_step(b, 2)
    P.lbm_step(b[1], 1)
    P.lbm_step(b[3], 1)
    P.lbm_batch_step(b, 1)
    got = _states(b)
    ref = _batch("f16", steps)
    P.lbm_batch_set_tile_shape(ref, shape)
    P.lbm_batch_step(ref, 2)
    for i in (1, 3):
        P.lbm_step(ref[i], 1)
    P.lbm_batch_step(ref, 1)
    for x, y in zip(got, _states(ref)):
        assert np.array_equal(x, y)
    other = _batch("f16", steps)
    P.lbm_batch_step(other, 2)
    for i in (1, 3):
        P.lbm_step(other[i], 1)
    P.lbm_batch_step(other, 1)
    for x, y in zip(got, _states(other)):
        assert np.abs(x - y).max() <= 1e-3 * np.abs(y).max()
    with pytest.raises(P.LbmError):
        P.lbm_batch_set_tile_shape(b, 1)


def test_direct_step_of_one_instance_between_replays():
    """Stepping an instance on its own changes its buffers and draw queue: the batch must
    notice and re-capture, so every instance still follows its own sequence of steps."""
    steps = 6
    b = _batch("f16", steps)
    P.lbm_batch_step(b, 2)
    P.lbm_step(b[2], 1)   # the forced instance: buffers and the head of its draw queue move
    P.lbm_step(b[0], 2)   # an unforced instance, an even number of steps: buffers unchanged
    P.lbm_batch_step(b, 2)
    got = _states(b)
    for i, n in enumerate([6, 4, 5, 4]):
        assert np.array_equal(got[i], _individual(i, "f16", steps, n)), f"instance {i}"


def test_batch_checks_its_arguments():
    with pytest.raises(P.LbmError):
        P.lbm_batch_create([dict(nx=8, ny=8, nz=8, nu=0.01, op="bgk")])
    with pytest.raises(P.LbmError):
        P.lbm_batch_create([dict(nx=8, ny=8, nz=8, nu=0.01, storage="f16"),
                            dict(nx=8, ny=8, nz=8, nu=0.01, storage="f32")])
    b = P.lbm_batch_create([dict(nx=8, ny=8, nz=8, nu=0.01, storage="f16")])
    with pytest.raises(P.LbmError):
        P.lbm_batch_step(b, 1)  # no weights yet
    P.lbm_batch_set_weights(b, G.theta0())
    f = P.lbm_batch_create([dict(nx=8, ny=8, nz=8, nu=0.01, storage="f16", forcing=dict(power=1e-6))])
    P.lbm_batch_set_weights(f, G.theta0())
    G.init_gpu(f[0], np.ones((8, 8, 8)), np.zeros((3, 8, 8, 8)))
    with pytest.raises(P.LbmError):
        P.lbm_batch_step(f, 1)  # no random draws queued
    with pytest.raises(ValueError):
        P.lbm_destroy(b[0])     # owned by the batch
    P.lbm_batch_destroy(b)


@pytest.mark.parametrize("weights", ["seed0", "sensitive"])
def test_batch_step_against_the_bf16_oracle(weights):
    """One batched step of instances of uneven size and viscosity from random populations,
    each instance against the BF16-operand oracle and its bound (tests/bf16_ref.py)."""
    from oracle import collision as col
    from tests import bf16_ref as B
    sizes = (27, 20, 20, 4)
    theta = B.case_theta(sizes, weights)
    specs = [((7, 6, 5), 0.02, 17), ((9, 17, 33), 0.004, 19), ((8, 8, 8), 0.01, 31)]
    b = P.lbm_batch_create([dict(nx=s[2], ny=s[1], nz=s[0], nu=nu, storage="f16") for s, nu, _ in specs])
    P.lbm_batch_set_weights(b, theta)
    starts = []
    for i, (shape, _, seed) in enumerate(specs):
        G.set_gpu_state(b[i], lbm_inputs.random_populations(shape, seed))
        starts.append(G.to_oracle_f(G.gpu_state(b[i])))
    P.lbm_batch_step(b, 1, use_graph=True)
    assert P.lbm_batch_check(b) == 0
    for i, (shape, nu, _) in enumerate(specs):
        got = G.to_oracle_f(G.gpu_state(b[i]))
        ref, bound = B.step_reference(starts[i], col.tau_from_nu(nu), theta.astype(np.float64), sizes)
        ok = B.within(got, ref, bound, "f16")
        assert ok.all(), (i, int((~ok).sum()), np.abs(got - ref).max())
