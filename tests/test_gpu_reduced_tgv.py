"""GPU tests of the reduced Taylor-Green domain of Appendix A ([0, pi/2]^3, boundary
"tgv_reduced"): the same step as the FP64 oracle's reduced domain, and the same flow as the
full periodic box run on the GPU and restricted to the domain (the paper's check at the end
of Appendix A), for every operator and for the tensor-core network."""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from oracle import lattice as L
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


def _fields(n_red, u0=0.05):
    rho, u = lbm_inputs.taylor_green_3d(4 * n_red, u0, shifted=True)
    return rho, u


@pytest.mark.parametrize("op", ["bgk", "kbc", "reg", "nco"])
def test_reduced_domain_one_step_parity_with_the_oracle(op):
    n, nu = 6, 0.01
    rho, u = _fields(n)
    theta = G.theta0()
    ctx = G.make_ctx((n, n, n), nu, op, bc="tgv_reduced", theta=theta)
    G.init_gpu(ctx, rho[:n, :n, :n], u[:, :n, :n, :n])
    P.lbm_step(ctx, 2)
    got = G.to_oracle_f(G.gpu_state(ctx))
    ref = G.oracle_sim_from_fields(rho[:n, :n, :n], u[:, :n, :n, :n], col.tau_from_nu(nu), op, theta=theta,
                                   bc="tgv_reduced").step(2).f
    assert G.rel_maxnorm(got, ref) <= 1e-5


@pytest.mark.parametrize("form", [("nco", "f32", "f32"), ("bgk", "f32", "f32"), ("nco", "f16", "bf16")])
def test_reduced_domain_equals_the_full_box_on_the_gpu(form):
    op, storage, net = form
    n, nu, steps = 8, 0.002, 40
    rho, u = _fields(n)
    theta = G.theta0()
    full = G.make_ctx((4 * n,) * 3, nu, op, storage=storage, net=net, theta=theta)
    red = G.make_ctx((n,) * 3, nu, op, storage=storage, net=net, bc="tgv_reduced", theta=theta)
    G.init_gpu(full, rho, u)
    G.init_gpu(red, rho[:n, :n, :n], u[:, :n, :n, :n])
    P.lbm_step(full, steps)
    P.lbm_step(red, steps)
    ff = G.gpu_state(full)[:, :n, :n, :n]
    fr = G.gpu_state(red)
    tol = 1e-6 if storage == "f32" else 1e-4
    assert np.abs(fr - ff).max() <= tol * np.abs(ff).max()
    # the box average of |u|^2 / 2 equals the domain average (the symmetries preserve |u|);
    # the two runs round differently (permuted arithmetic, and 16-bit storage in the mixed form)
    assert P.lbm_kinetic_energy(red) == pytest.approx(P.lbm_kinetic_energy(full), rel=tol * 10)


def test_reduced_domain_state_roundtrip_and_refusals():
    n = 5
    ctx = G.make_ctx((n, n, n), 0.01, "bgk", bc="tgv_reduced")
    f0 = lbm_inputs.random_populations((n, n, n), 7)
    G.set_gpu_state(ctx, f0)
    # the pull map is a bijection on the reduced domain too: set/get are inverses (up to the
    # FP32 rounding of the stored deviations f - w)
    w = L.W[:, None, None, None]
    assert np.abs(G.gpu_state(ctx) - f0).max() <= 2.0 ** -24 * (np.abs(f0 - w).max() + 2 * np.abs(f0).max())
    with pytest.raises(P.LbmError):
        P.lbm_energy_spectrum(ctx, torch.zeros(n + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(P.LbmError):
        P.lbm_create(4, 4, 6, 0.01, boundary="tgv_reduced")   # not a cube
    with pytest.raises(P.LbmError):  # spectral forcing needs the periodic box
        P.lbm_create(n, n, n, 0.01, op="bgk", boundary="tgv_reduced", forcing=dict(power=1e-6))
    # recording for the adjoint covers the reduced domain with the FP32 network
    # (tests/test_gpu_adjoint_dissipation.py), not the tensor-core forms
    P.lbm_record_begin(G.make_ctx((n, n, n), 0.01, "nco", bc="tgv_reduced", theta=G.theta0()), 2)
    tc = G.make_ctx((n, n, n), 0.01, "nco", storage="f16", net="bf16", bc="tgv_reduced", theta=G.theta0())
    with pytest.raises(P.LbmError):
        P.lbm_record_begin(tc, 2)
