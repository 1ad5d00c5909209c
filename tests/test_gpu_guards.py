"""Guard regions around the population buffers (lbm_check_guards), the check of
out-of-bounds writes that stands in for a sanitizer: every step, init and state kernel, on
ragged grids and every boundary, storage and network form, leaves the four 4 KB regions
before and after the two buffers untouched, and a changed guard byte is reported
(lbm_selftest_guards changes one with a memset of the context's own allocation)."""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [  # shape (nz, ny, nx), op, storage, net, boundary, forced
    ((5, 6, 7), "bgk", "f32", "f32", "periodic", False),
    ((5, 6, 7), "kbc", "f16", "f32", "mirror", False),
    ((7, 6, 5), "nco", "f16", "bf16", "periodic", True),
    ((7, 6, 5), "nco", "bf16", "bf16", "mirror", False),
    ((9, 17, 33), "nco", "f32", "bf16x3", "periodic", True),
    ((4, 5, 6), "nco", "f32", "f32", "periodic", True),
    ((8, 8, 8), "reg", "bf16", "f32", "tgv_reduced", False),
    ((1, 1, 1), "bgk", "f16", "f32", "periodic", False),
]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(str(v) for v in c[1:]) + f"-{c[0]}")
def test_guard_regions_stay_intact(case):
    shape, op, storage, net, bc, forced = case
    ctx = G.make_ctx(shape, 0.01, op, storage=storage, net=net, bc=bc, theta=G.theta0(),
                     forcing=dict(power=1e-6) if forced else None)
    P.lbm_check_guards(ctx)
    rng = np.random.default_rng(3)
    G.init_gpu(ctx, 1.0 + 0.01 * rng.standard_normal(shape), 0.02 * rng.standard_normal((3,) + shape))
    if forced:
        phi, psi = lbm_inputs.forcing_draws(6, seed=2)
        P.lbm_force_draws(ctx, phi, psi)
    P.lbm_step(ctx, 1)
    P.lbm_step(ctx, 5)
    f = torch.empty((27,) + shape, dtype=torch.float32, device="cuda")
    P.lbm_get_state(ctx, f)
    P.lbm_set_state(ctx, f)
    assert P.lbm_check(ctx) == 0
    P.lbm_check_guards(ctx)
    P.lbm_selftest_guards(ctx)
    P.lbm_check_guards(ctx)
    P.lbm_destroy(ctx)
