"""Parity at the full size of the throughput workload (the Re-1600 Taylor-Green vortex on
256^3, initialised as bench.py does), in the launch configuration bench.py times (one
step kernel over the whole grid per lbm_step), for every form the bench reports.

The FP64 oracle cannot step 16.8 M cells, so it checks sampled outputs one by one: for a
sampled cell x, f_i(x, t+1) = C(f(x - c_i, t))_i, and the oracle applies its collision C
to the GPU's own pre-step populations of the 27 source cells. Samples: the eight corners,
face and edge cells (periodic wrap), both sides of 128-cell tile boundaries, and random
cells. Properties that hold at any size are checked on the whole grid: total mass and
momentum are conserved by the step.

Tolerances as at small sizes: FP32 storage with the FP32 or split-BF16 network 1e-5
relative (the split form adds 1e-4 x the higher-order part its rates act on); the mixed
form against the BF16-operand oracle and its bound (tests/bf16_ref.py), the stored FP16
deviation being a rounding of a value within that bound. The mixed form is also checked
on random populations far from equilibrium over the whole 256^3 grid, with the seed-0 and
the state-sensitive weights, where the rates act on a large higher-order part.
"""

import numpy as np
import pytest

import lbm_inputs
import paper_2412_08229_gb300 as P
from oracle import collision as col
from oracle import lattice as L
from tests import bf16_ref as B
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, U0, RE = 256, 0.05, 1600.0
FORMS = {  # name: (operator, storage, network)
    "mixed": ("nco", "f16", "bf16"),
    "fp32_tc3": ("nco", "f32", "bf16x3"),
    "fp32": ("nco", "f32", "f32"),
    "bgk_f32": ("bgk", "f32", "f32"),
    "kbc_f32": ("kbc", "f32", "f32"),
    "bgk_f16": ("bgk", "f16", "f32"),
}
RATE_TOL = {"bf16x3": 1e-4, "f32": 0.0}
HALF_ULP = {"f32": 2.0 ** -24, "f16": 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P._abi.load()


@pytest.fixture(scope="module")
def fields():
    return lbm_inputs.taylor_green_3d(N, U0)


def _samples():
    """(x, y, z) of the sampled cells."""
    pts = set()
    for x in (0, N - 1):
        for y in (0, N - 1):
            for z in (0, N - 1):
                pts.add((x, y, z))
    for t in (0, 1, 127, 128, 129, 255):  # tile boundaries along x (tiles are 128 cells of one row)
        pts.add((t, 0, 0))
        pts.add((t, 17, 200))
    for e in range(N // 32):
        pts.add((0, 32 * e, N - 1))
        pts.add((N - 1, 5, 32 * e))
    rng = np.random.default_rng(12)
    while len(pts) < 160:
        pts.add(tuple(int(v) for v in rng.integers(0, N, 3)))
    return np.array(sorted(pts), dtype=np.int64)


def _gather(f, xyz):
    """Populations (k, 27) float64 at cells (x, y, z) of a (27, N, N, N) = (27, z, y, x) tensor."""
    idx = torch.from_numpy(xyz).cuda()
    return f[:, idx[:, 2], idx[:, 1], idx[:, 0]].T.double().cpu().numpy()


def _collide(op, f, tau, theta, net="f32"):
    if op == "bgk":
        return col.bgk(f, tau)
    if op == "kbc":
        return col.kbc_collide(f, tau)
    if net == "bf16":
        return col.mrt_collide(f, tau, B.rates(f, theta))
    return col.nco_collide(f, tau, theta)


def _higher_order_part(f):
    m = col.moments(f)
    mh = np.where(L.MOMENT_ORDER >= 3, m, 0.0)
    return float(np.abs(mh @ L.M_INV.T).max())


def _totals(ctx):
    rho = torch.empty((N, N, N), device="cuda")
    u = torch.empty((3, N, N, N), device="cuda")
    P.lbm_macroscopic(ctx, rho, u)
    r = rho.double()
    return float(r.sum()), (u.double() * r).sum(dim=(1, 2, 3)).cpu().numpy(), float((u.double().abs() * r).sum())


@pytest.mark.parametrize("form", list(FORMS))
def test_full_size_step_on_sampled_cells(form, fields):
    op, storage, net = FORMS[form]
    rho, u = fields
    nu = lbm_inputs.reynolds_viscosity(U0, N, RE)
    tau = col.tau_from_nu(nu)
    theta = G.theta0()
    ctx = P.lbm_create(N, N, N, nu, op=op, storage=storage, net=net)
    try:
        if op == "nco":
            P.nco_set_weights(ctx, torch.from_numpy(theta).cuda())
        P.lbm_init(ctx, torch.from_numpy(rho.astype(np.float32)).cuda(), torch.from_numpy(u.astype(np.float32)).cuda())
        P.lbm_step(ctx, 3)  # leave the equilibrium start: non-equilibrium moments present
        mass0, mom0, scale0 = _totals(ctx)
        f = torch.empty((27, N, N, N), device="cuda")
        P.lbm_get_state(ctx, f)
        xyz = _samples()
        # the 27 source cells of every sample, x - c_i with periodic wrap
        src = (xyz[:, None, :] - L.C[None, :, :]) % N                  # (k, 27, 3)
        uniq, inv = np.unique(src.reshape(-1, 3), axis=0, return_inverse=True)
        f_src = _gather(f, uniq)
        post = _collide(op, f_src, tau, theta.astype(np.float64), net)  # (u, 27)
        ref = post[inv.reshape(-1, 27), np.arange(27)[None, :]]        # (k, 27)
        if net == "bf16":
            pb = B.population_bound(f_src, B.rate_bound(f_src, theta.astype(np.float64)))
            bound = pb[inv.reshape(-1, 27), np.arange(27)[None, :]]
        P.lbm_step(ctx, 1)
        assert P.lbm_check(ctx) == 0
        P.lbm_get_state(ctx, f)
        got = _gather(f, xyz)
        mass1, mom1, _ = _totals(ctx)
    finally:
        P.lbm_destroy(ctx)
        torch.cuda.empty_cache()
    if net == "bf16":
        ok = B.within(got, ref, bound, storage)
        assert ok.all(), (form, int((~ok).sum()), np.abs(got - ref).max())
    else:
        tol = (RATE_TOL[net] * _higher_order_part(f_src) + HALF_ULP[storage] * np.abs(ref - L.W).max()
               + 1e-5 * np.abs(ref).max())
        assert np.abs(got - ref).max() <= tol, (form, np.abs(got - ref).max(), tol)
    # whole-grid conservation of the step (periodic box)
    assert abs(mass1 - mass0) <= 1e-6 * mass0
    assert np.abs(mom1 - mom0).max() <= 1e-6 * scale0


@pytest.mark.parametrize("weights", ["seed0", "sensitive"])
def test_full_size_mixed_step_on_random_populations(weights):
    """The mixed form at 256^3 in the bench's launch configuration from random populations
    (uniform in [0.01, 0.05), far from equilibrium) on every cell, sampled cells against
    the BF16-operand oracle and its bound."""
    theta = B.case_theta((27, 20, 20, 4), weights)
    nu = lbm_inputs.reynolds_viscosity(U0, N, RE)
    tau = col.tau_from_nu(nu)
    ctx = P.lbm_create(N, N, N, nu, op="nco", storage="f16", net="bf16")
    try:
        P.nco_set_weights(ctx, torch.from_numpy(theta).cuda())
        f0 = lbm_inputs.random_populations((N, N, N), 23).astype(np.float32)
        f = torch.from_numpy(f0).cuda()
        del f0
        P.lbm_set_state(ctx, f)
        P.lbm_get_state(ctx, f)
        xyz = _samples()
        src = (xyz[:, None, :] - L.C[None, :, :]) % N
        uniq, inv = np.unique(src.reshape(-1, 3), axis=0, return_inverse=True)
        f_src = _gather(f, uniq)
        th = theta.astype(np.float64)
        post = col.mrt_collide(f_src, tau, B.rates(f_src, th))
        pb = B.population_bound(f_src, B.rate_bound(f_src, th))
        pick = (inv.reshape(-1, 27), np.arange(27)[None, :])
        ref, bound = post[pick], pb[pick]
        P.lbm_step(ctx, 1)
        assert P.lbm_check(ctx) == 0
        P.lbm_get_state(ctx, f)
        got = _gather(f, xyz)
    finally:
        P.lbm_destroy(ctx)
        torch.cuda.empty_cache()
    ok = B.within(got, ref, bound, "f16")
    assert ok.all(), (int((~ok).sum()), np.abs(got - ref).max())
