"""The spectrum's shell of every wave vector, as the library's device binning code computes
it, equals the oracle's integer shell rule (oracle.diagnostics.shell_index: the n with
n^2 - n + 1 <= |k|^2 <= n^2 + n) bit for bit, up to the 256^3 box of the headline workload
and on odd and mixed box sizes."""

import numpy as np
import pytest

import paper_2412_08229_gb300 as P
from oracle import diagnostics as D

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


@pytest.mark.parametrize("shape", [(256, 256, 256), (64, 64, 64), (7, 12, 15), (1, 1, 2048), (96, 48, 32)])
def test_shell_indices_bit_exact(shape):
    nz, ny, nx = shape
    got = P.lbm_spectrum_shells(nx, ny, nz)
    kz, ky, kx = np.meshgrid(D.wavenumbers(nz), D.wavenumbers(ny), D.wavenumbers(nx), indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    table = D.shell_index(np.arange(int(k2.max()) + 1))   # the oracle's rule for every integer |k|^2
    assert np.array_equal(got, table[k2].astype(np.int32))
