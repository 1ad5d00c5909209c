"""CPU checks of the BF16 network's parity tolerance (tests/bf16_ref.py): the reference
rounds operands as the kernels do, its bound covers the rounding ambiguities it is meant
to cover, and the check rejects plausible kernel mistakes on the very inputs of the GPU
parity tests (mistakes are planted in the oracle, on the CPU):
  * the network replaced by its cell-mean constant rates (a kernel that ignores the state);
  * the group action dropped (the network applied to m alone, no average over O_h);
  * the group table with its signs dropped (a wrong W1 P_g image);
  * two third-order moments swapped in the network input (a wrong A1 layout).
With the seed-0 Kaiming weights the rates vary little with the state (their spread over
random cells is below 0.01), so the subtle last mistake moves them by only about twice
the bound and 16-bit storage rounding hides it for the deeper network; the GPU tests
therefore also run every case with state-sensitive weights (W1 x 30), which must reject
all four mistakes in every storage format.
"""

import numpy as np
import pytest

import lbm_inputs
from oracle import collision as col
from oracle import lattice as L
from tests import bf16_ref as B

STORAGES = ("f32", "f16", "bf16")


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 1.001953125, 3.0e-39, -2.5]])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(B.bf16(x), want)
    normal = np.abs(x) >= 2.0 ** -126
    err = np.abs(B.bf16(x) - x.astype(np.float32).astype(np.float64))[normal]
    assert np.all(err <= 0.5 * B.ulp_bf16(x.astype(np.float32))[normal])


def _f(case):
    shape, seed = B.CASES[case][0], B.CASES[case][1]
    return np.moveaxis(lbm_inputs.random_populations(shape, seed), 0, -1)


@pytest.mark.parametrize("weights", ["seed0", "sensitive"])
def test_table_form_equals_the_oracle_network(weights):
    sizes = col.LAYER_SIZES
    theta = B.case_theta(sizes, weights).astype(np.float64)
    f = _f("ragged").reshape(-1, 27)
    exact = col.nco_rates(f, theta)
    assert np.allclose(B.rates_with_table(f, theta, operand_round=None), exact, rtol=0, atol=1e-13)
    assert np.allclose(B.rates_with_table(f, theta), B.rates(f, theta), rtol=0, atol=1e-13)


@pytest.mark.parametrize("case", list(B.CASES))
@pytest.mark.parametrize("weights", ["seed0", "sensitive"])
def test_bound_covers_one_input_flip(case, weights):
    """Moving any one BF16 input of a cell to its neighbour moves every rate by less than
    half the bound (the bound allows two flips and a factor 2 for ReLU kinks)."""
    sizes = B.CASES[case][3]
    theta = B.case_theta(sizes, weights).astype(np.float64)
    f = _f(case).reshape(-1, 27)[:400]
    m = col.moments(f)
    mb = B.bf16(m)
    base = B.rates_from_moments(mb, theta, sizes)
    tol = B.rate_bound(f, theta, sizes)
    worst = 0.0
    for k in range(27):
        for d in (1.0, -1.0):
            moved = mb.copy()
            moved[:, k] += d * B.ulp_bf16(mb[:, k])
            worst = max(worst, float((np.abs(B.rates_from_moments(moved, theta, sizes) - base) / tol).max()))
    assert worst <= 0.5, worst


def _stored_step(start, tau, rates, bc, storage):
    post = col.mrt_collide(start, tau, rates)
    dev = B.storage_round(post - L.W, storage)
    return B.stream((dev.astype(np.float32) + L.W.astype(np.float32)).astype(np.float64), bc)


def _swap_two_third_order():
    k3 = np.where(L.MOMENT_ORDER == 3)[0]
    sw = np.arange(27)
    sw[k3[0]], sw[k3[3]] = k3[3], k3[0]
    return sw


MISTAKES = {  # name: (table or None for constant rates, caught with the seed-0 weights too)
    "constant rates": (None, True),
    "no group average": ((np.tile(np.arange(27), (L.G, 1)), np.ones((L.G, 27), dtype=np.int64)), True),
    "group signs dropped": ((B._PERM, np.abs(B._SIGN)), True),
    "input layout": ((B._PERM[:, _swap_two_third_order()], B._SIGN[:, _swap_two_third_order()]), False),
}


@pytest.mark.parametrize("case", list(B.CASES))
@pytest.mark.parametrize("weights", ["seed0", "sensitive"])
def test_tolerance_accepts_the_reference_and_rejects_planted_mistakes(case, weights):
    shape, seed, nu, sizes, bcs = B.CASES[case]
    theta = B.case_theta(sizes, weights).astype(np.float64)
    tau = col.tau_from_nu(nu)
    f0 = lbm_inputs.random_populations(shape, seed)
    for storage in STORAGES:
        start = B.stored_start(f0, storage)
        flat = start.reshape(-1, 27)
        w_ref = B.rates(flat, theta, sizes)
        for bc in bcs:
            ref, bound = B.step_reference(start, tau, theta, sizes, bc)
            ok = _stored_step(start, tau, w_ref.reshape(shape + (4,)), bc, storage)
            assert B.within(ok, ref, bound, storage).all(), (storage, bc)
            for name, (table, gross) in MISTAKES.items():
                if weights == "seed0" and not gross:
                    continue
                if table is None:
                    bad_rates = np.broadcast_to(w_ref.mean(axis=0), w_ref.shape)
                else:
                    bad_rates = B.rates_with_table(flat, theta, sizes, table)
                bad = _stored_step(start, tau, bad_rates.reshape(shape + (4,)), bc, storage)
                frac = 1.0 - B.within(bad, ref, bound, storage).mean()
                assert frac > 0.0, (name, storage, bc)
