"""The allocation-free kinetic-energy entry point agrees with the FP64 oracle's kinetic
energy (oracle.diagnostics.kinetic_energy of the oracle's macroscopic velocity) and with
the context-based entry point, on two calls in a row, up to the largest grid its scratch
serves (256^3 cells: all 4096 partial sums).

lbm_kinetic_energy_noalloc exists for callers that may not allocate device memory
(for example code whose every device byte comes from a host framework's pool); it keeps
its reduction scratch in a fixed array inside the library. This file is collected
last so that a run stopping at the first failure has already run every other test;
it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from oracle import diagnostics as D
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def test_noalloc_kinetic_energy_matches_context_path_twice():
    torch = G.torch_cuda()
    shape = (19, 18, 17)  # 5814 cells: two blocks of the reduction, the second partial
    nz, ny, nx = shape
    f = lbm_inputs.random_populations(shape, 51)
    ctx = G.make_ctx(shape, 0.02, "bgk")
    G.set_gpu_state(ctx, f)
    ref = P.lbm_kinetic_energy(ctx)
    oracle = D.kinetic_energy(col.macroscopic(G.to_oracle_f(f.astype(np.float32)))[1])
    assert ref == pytest.approx(oracle, rel=1e-5)
    f_dev = torch.from_numpy(f.astype(np.float32)).cuda()
    for _ in range(2):  # the shared scratch keeps the last call's contents
        ke = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        P.lbm_kinetic_energy_noalloc(f_dev, nx, ny, nz, ke)
        torch.cuda.synchronize()
        assert float(ke.item()) == pytest.approx(oracle, rel=1e-5)
        assert float(ke.item()) == pytest.approx(ref, rel=1e-5)
    # a smaller grid after a larger one reads only the partial sums it wrote
    small = f_dev[:, :2].contiguous()
    ctx2 = G.make_ctx((2, ny, nx), 0.02, "bgk")
    G.set_gpu_state(ctx2, f[:, :2].copy())
    ke = torch.zeros(1, dtype=torch.float64, device="cuda")
    P.lbm_kinetic_energy_noalloc(small, nx, ny, 2, ke)
    torch.cuda.synchronize()
    assert float(ke.item()) == pytest.approx(P.lbm_kinetic_energy(ctx2), rel=1e-5)


def test_noalloc_at_its_largest_grid_matches_the_oracle_twice():
    """256^3 cells, exactly the 4096 partial sums of the scratch: per-cell velocities in
    FP32 from FP32 populations, (1/2)|u|^2 summed in FP64; relative error well below 1e-5."""
    torch = G.torch_cuda()
    n = 256
    f = lbm_inputs.random_populations((n, n, n), 53).astype(np.float32)
    _, u = col.macroscopic(np.moveaxis(f, 0, -1).astype(np.float64))
    oracle = D.kinetic_energy(u)
    del u
    f_dev = torch.from_numpy(f).cuda()
    del f
    for _ in range(2):
        ke = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        P.lbm_kinetic_energy_noalloc(f_dev, n, n, n, ke)
        torch.cuda.synchronize()
        assert float(ke.item()) == pytest.approx(oracle, rel=1e-5)
    del f_dev
    torch.cuda.empty_cache()


def test_noalloc_rejects_grids_beyond_its_scratch_and_host_pointers():
    torch = G.torch_cuda()
    f = torch.zeros(27, dtype=torch.float32, device="cuda")
    ke = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(P.LbmError) as e:
        P.lbm_kinetic_energy_noalloc(f, 257, 256, 256, ke)  # more cells than 4096 partials of 4096
    assert e.value.status == P._abi.LBM_ERR_ARG
    with pytest.raises(P.LbmError) as e:
        P.lbm_kinetic_energy_noalloc(np.zeros(27, np.float32), 1, 1, 1, ke)  # host input
    assert e.value.status == P._abi.LBM_ERR_ARG
