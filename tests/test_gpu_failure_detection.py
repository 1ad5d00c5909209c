"""Failure detection of the tensor-core step kernels, without a GPU fault.

Every wait of these kernels on MMA completion is bounded. lbm_set_wait_limit shortens the
main waits of one context (0: give up at the first one), so the step kernel stops early
and latches a status flag that lbm_check reports as LBM_ERR_TIMEOUT. Before it releases
its tensor memory the kernel still waits, with the full limit, for the MMAs it had
started; the message of lbm_check says whether that drain succeeded. The GPU stays usable:
a fresh context steps correctly afterwards and the tensor-core self-test is still exact.
"""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def _tgv_ctx(net, storage):
    shape = (16, 16, 16)
    ctx = G.make_ctx(shape, 0.01, "nco", storage=storage, net=net, theta=G.theta0())
    G.init_gpu(ctx, *lbm_inputs.taylor_green_3d(16, 0.05))
    return ctx


@pytest.mark.parametrize("net,storage", [("bf16", "f16"), ("bf16", "f32"), ("bf16x3", "f32")])
def test_timed_out_mma_wait_is_reported_latched_and_drained(net, storage):
    ctx = _tgv_ctx(net, storage)
    P.lbm_set_wait_limit(ctx, 0)
    P.lbm_step(ctx, 2)  # asynchronous: the flag is read by lbm_check
    for _ in range(2):  # latched
        with pytest.raises(P.LbmError) as e:
            P.lbm_check(ctx)
        assert e.value.status == P._abi.LBM_ERR_TIMEOUT
        assert "ran out" in str(e.value) and "left allocated" not in str(e.value)
    P.lbm_destroy(ctx)
    torch.cuda.synchronize()
    # the device is usable: a fresh context with the default limit steps correctly
    fresh = _tgv_ctx(net, storage)
    f0 = lbm_inputs.random_populations((16, 16, 16), 61)
    G.set_gpu_state(fresh, f0)
    start = G.to_oracle_f(G.gpu_state(fresh))
    P.lbm_step(fresh, 1)
    assert P.lbm_check(fresh) == 0
    got = G.to_oracle_f(G.gpu_state(fresh))
    if net == "bf16":
        from tests import bf16_ref as B
        ref, bound = B.step_reference(start, col.tau_from_nu(0.01), G.theta0().astype(np.float64))
        assert B.within(got, ref, bound, storage).all()
    else:
        from oracle import stepper as S
        ref = S.Simulation(start, col.tau_from_nu(0.01), op="nco", theta=G.theta0().astype(np.float64)).step(1).f
        assert G.rel_maxnorm(got, ref) <= 1e-4
    assert P.lbm_selftest_tensor_cores() == 0.0


def test_wait_limit_argument_is_checked():
    ctx = _tgv_ctx("bf16", "f16")
    with pytest.raises(P.LbmError) as e:
        P.lbm_set_wait_limit(ctx, -1)
    assert e.value.status == P._abi.LBM_ERR_ARG
    P.lbm_set_wait_limit(ctx, 2_000_000_000)  # the default: steps run normally
    P.lbm_step(ctx, 3)
    assert P.lbm_check(ctx) == 0
