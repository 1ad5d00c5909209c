"""GPU parity of the network with a third hidden layer (27-20-20-20-4, 1484 parameters;
the deeper variant the paper also trains, Sec. IV) against the FP64 oracle, which takes
the layer sizes as a parameter.

FP32 network: 1e-5 relative after one step, as for the two-layer network. BF16 tensor-core
network: the BF16-operand oracle and its bound (tests/bf16_ref.py, which follows the
rounding through every hidden layer), with the seed-0 and the state-sensitive weights.
"""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from oracle import stepper as S
from tests import bf16_ref as B
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIZES = (27, 20, 20, 20, 4)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def _theta():
    return lbm_inputs.nco_parameters(0, SIZES).astype(np.float32)


def test_deep_network_parameter_count():
    assert _theta().size == 1484


@pytest.mark.parametrize("bc", ["periodic", "mirror"])
def test_deep_fp32_network_one_step(bc):
    shape = (7, 6, 5)
    f0 = lbm_inputs.random_populations(shape, 41)
    nu = 0.02
    theta = _theta()
    ctx = G.make_ctx(shape, nu, "nco", bc=bc, theta=theta)
    G.set_gpu_state(ctx, f0)
    start = G.to_oracle_f(G.gpu_state(ctx))
    P.lbm_step(ctx, 1)
    got = G.to_oracle_f(G.gpu_state(ctx))
    ref = S.Simulation(start, col.tau_from_nu(nu), op="nco", theta=theta.astype(np.float64), bc=bc,
                       sizes=SIZES).step(1).f
    assert G.rel_maxnorm(got, ref) <= 1e-5


@pytest.mark.parametrize("weights", ["seed0", "sensitive"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_deep_bf16_network_one_step(storage, weights):
    shape, seed, nu, sizes, _ = B.CASES["deep"]
    theta = B.case_theta(sizes, weights)
    ctx = G.make_ctx(shape, nu, "nco", storage=storage, net="bf16", theta=theta)
    G.set_gpu_state(ctx, lbm_inputs.random_populations(shape, seed))
    G.check_bf16_step(ctx, nu, theta, sizes, "periodic", storage)


def test_deep_network_tgv16_fp32_and_bf16():
    rho, u = lbm_inputs.taylor_green_3d(16, 0.05)
    nu = 0.005
    theta = _theta()
    a = G.make_ctx((16,) * 3, nu, "nco", net="f32", theta=theta)
    b = G.make_ctx((16,) * 3, nu, "nco", storage="f16", net="bf16", theta=theta)
    for c in (a, b):
        G.init_gpu(c, rho, u)
    P.lbm_step(a, 2)
    ref = G.oracle_sim_from_fields(rho, u, col.tau_from_nu(nu), "nco", theta=theta, sizes=SIZES).step(2).f
    assert G.rel_maxnorm(G.to_oracle_f(G.gpu_state(a)), ref) <= 1e-5
    for _ in range(2):  # each step from the state the GPU reached
        G.check_bf16_step(b, nu, theta, SIZES, "periodic", "f16")


def test_deep_network_is_refused_where_not_covered():
    ctx = G.make_ctx((8, 8, 8), 0.01, "nco", theta=_theta())
    P.lbm_record_begin(ctx, 2)  # the adjoint covers both depths (tests/test_gpu_adjoint_dissipation.py)
    b = P.lbm_batch_create([dict(nx=8, ny=8, nz=8, nu=0.01, storage="f16")])
    with pytest.raises(P.LbmError):
        P.lbm_batch_set_weights(b, _theta())
    with pytest.raises(P.LbmError):
        P.nco_set_weights(ctx, np.zeros(1000, dtype=np.float32))
