"""Recording and adjoint buffers come from the library's per-device stream-ordered pool,
which keeps released memory for reuse; destroying the context gives it back to the device."""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def _free():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


def _train_once(n, steps):
    ctx = G.make_ctx((n, n, n), 0.01, "nco", theta=G.theta0())
    G.init_gpu(ctx, *lbm_inputs.taylor_green_3d(n, 0.05))
    P.lbm_record_begin(ctx, 1)
    P.lbm_step(ctx, steps)
    grad = np.zeros(1064, dtype=np.float32)
    du = np.ones((3, n, n, n), dtype=np.float32)
    P.nco_backward(ctx, du, None, grad, None)
    return ctx


def test_destroy_returns_recording_memory_to_the_device():
    n, steps = 64, 12
    P.lbm_destroy(_train_once(16, 2))  # first use: pool creation, module loads
    free0 = _free()
    ctx = _train_once(n, steps)
    held = free0 - _free()
    state = n ** 3 * 27 * 4
    assert held >= (steps + 1) * state  # one checkpoint per step, kept in the pool
    P.lbm_destroy(ctx)
    assert free0 - _free() <= 16 * 2 ** 20, "memory of the destroyed context still reserved"
