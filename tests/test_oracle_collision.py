"""Pins of oracle.collision: closed forms, conservation, reductions, invariance (CPU only)."""

import numpy as np
import pytest

import lbm_inputs
from oracle import collision as col
from oracle import lattice as L
from tests.conftest import read_golden


def _random_state(n, seed, amp=0.08):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.9, 1.1, size=n)
    u = rng.uniform(-amp, amp, size=(n, 3))
    return rho, u


def _random_f(n, seed):
    return lbm_inputs.random_populations((n,), seed).T.copy()  # (n, 27)


def test_equilibrium_moments_closed_form():
    """m^eq = (rho, sqrt3 rho u, 3 rho u_a u_b, 0, ..., 0) for the quadratic f^eq."""
    rho, u = _random_state(50, 1)
    meq = col.equilibrium_moments(rho, u)
    s3 = np.sqrt(3.0)
    exp = np.zeros((50, 27))
    exp[:, 0] = rho
    exp[:, 1:4] = s3 * rho[:, None] * u
    pairs = {"xx": (0, 0), "xy": (0, 1), "xz": (0, 2), "yy": (1, 1), "yz": (1, 2), "zz": (2, 2)}
    for k, name in enumerate(L.MOMENT_NAMES):
        if name in pairs:
            a, b = pairs[name]
            exp[:, k] = 3.0 * rho * u[:, a] * u[:, b]
    assert np.allclose(meq, exp, atol=1e-14)


def test_equilibrium_reproduces_its_macroscopic_moments():
    rho, u = _random_state(40, 2)
    r2, u2 = col.macroscopic(col.equilibrium(rho, u))
    assert np.allclose(r2, rho, atol=1e-14) and np.allclose(u2, u, atol=1e-14)


def test_tau_viscosity_relation():
    assert col.tau_from_nu(0.005) == pytest.approx(0.515)
    assert col.tau_from_nu(0.0015) == pytest.approx(0.5045)


@pytest.mark.parametrize("op", ["bgk", "kbc", "reg", "nco"])
def test_collisions_conserve_mass_and_momentum(op):
    f = _random_f(64, 5)
    theta = lbm_inputs.nco_parameters(0)
    tau = 0.53
    if op == "bgk":
        fs = col.bgk(f, tau)
    elif op == "kbc":
        fs = col.kbc_collide(f, tau)
    elif op == "reg":
        fs = col.reg_collide(f, tau)
    else:
        fs = col.nco_collide(f, tau, theta)
    c = L.C.astype(float)
    assert np.allclose(fs.sum(-1), f.sum(-1), rtol=1e-14, atol=0)
    assert np.allclose(fs @ c, f @ c, rtol=0, atol=1e-15)


def test_mrt_with_all_rates_one_over_tau_is_bgk():
    f = _random_f(64, 6)
    tau = 0.61
    rates = np.full((64, 4), 1.0 / tau)
    assert np.allclose(col.mrt_collide(f, tau, rates), col.bgk(f, tau), atol=1e-15)


def test_kbc_with_gamma_two_is_bgk():
    f = _random_f(64, 7)
    assert np.allclose(col.kbc_collide(f, 0.57, gamma_override=2.0), col.bgk(f, 0.57), atol=1e-15)


def test_kbc_gamma_is_entropic_stationary_point():
    """KBC chooses gamma minimising the quadratic entropy proxy <f*-feq | f*-feq>_feq along Dh.

    With Ds and Dh fixed, <Dpost|Dpost> for Dpost = (1-2b) Ds + (1-b g) Dh is a
    parabola in g whose minimum is the published gamma.
    """
    f = _random_f(8, 8)
    tau = 0.52
    rho, u = col.macroscopic(f)
    feq = col.equilibrium(rho, u)
    fstar = col.kbc_collide(f, tau)
    for dg in (-1e-3, 1e-3):
        # perturbing gamma: f*(g + dg) = f*(g) - beta dg Dh
        dm = col.moments(f) - col.moments(feq)
        dh = np.where(L.MOMENT_ORDER >= 3, dm, 0.0) @ L.M_INV.T
        beta = 1.0 / (2.0 * tau)
        d0 = ((fstar - feq) ** 2 / feq).sum(-1)
        d1 = ((fstar - beta * dg * dh - feq) ** 2 / feq).sum(-1)
        assert (d1 >= d0 - 1e-18).all()


def test_network_architecture_and_parameter_count():
    rows = read_golden("nco_architecture.txt")
    for row in rows:
        sizes_s, count = row.split(";")
        sizes = tuple(int(v) for v in sizes_s.split())
        theta = lbm_inputs.nco_parameters(0, sizes)
        assert theta.size == int(count)
        assert len(col.unpack_theta(theta, sizes)) == len(sizes) - 1


def test_sigmoid_keeps_tau_in_half_open_interval():
    t = np.linspace(-30, 30, 1001)  # beyond |30| FP64 rounds to the interval ends
    tau = col.tau_from_network(t)
    assert (tau > 0.5).all() and (tau < 1.0).all()
    assert col.tau_from_network(np.array(0.0)) == pytest.approx(0.75)
    # literal sign of the printed sigmoid: large tau~ drives tau_n to 1/2 (rate 2)
    assert col.tau_from_network(np.array(30.0)) == pytest.approx(0.5, abs=1e-12)


def test_network_invariance_under_all_48_group_elements():
    """N_Phi(Pi_i f) = N_Phi(f) for every i in O_h (Sec. II.B)."""
    f = _random_f(32, 9)
    theta = lbm_inputs.nco_parameters(0)
    base = col.invariant_network(f, theta)
    for g in range(48):
        other = col.invariant_network(f[:, L.G_VPERM[g]], theta)
        assert np.allclose(other, base, rtol=0, atol=1e-13)


def test_network_group_average_closed_form_on_first_order_moments():
    """A network that reads one first-order moment averages relu over all signed axes.

    With W1 picking m_x only, W2 = identity on that unit and W3 summing it, the
    group average of relu(m_x^(g)) over O_h is (1/6) sum_a |m_a| because every
    signed axis +-a occurs 8 times among the 48 elements. A wrong group table or
    moment action breaks this closed form.
    """
    sizes = (27, 20, 20, 4)
    layers = [np.zeros((20, 27)), np.zeros(20), np.zeros((20, 20)), np.zeros(20),
              np.zeros((4, 20)), np.zeros(4)]
    layers[0][0, 1] = 1.0  # unit 0 reads m_x
    layers[2][0, 0] = 1.0
    layers[4][:, 0] = 1.0
    theta = np.concatenate([a.ravel() for a in layers])
    f = _random_f(16, 10)
    m = col.moments(f)
    out = col.invariant_network(f, theta, sizes)
    exp = np.abs(m[:, 1:4]).sum(axis=1) / 6.0
    for n in range(4):
        assert np.allclose(out[:, n], exp, atol=1e-14)


def test_network_with_zero_first_layers_is_constant():
    theta = lbm_inputs.nco_parameters(0).copy()
    layers = col.unpack_theta(theta)
    W1, b1 = layers[0]
    W1[...] = 0.0
    (W2, b2), (W3, b3) = layers[1], layers[2]
    f = _random_f(4, 11)
    out = col.invariant_network(f, theta)
    h = np.maximum(W2 @ np.maximum(b1, 0) + b2, 0)
    assert np.allclose(out, (W3 @ h + b3)[None, :], atol=1e-15)


@pytest.mark.parametrize("op", ["nco", "kbc", "reg", "bgk"])
def test_collision_equivariance_per_cell(op):
    f = _random_f(16, 12)
    theta = lbm_inputs.nco_parameters(0)
    fn = {"bgk": lambda x: col.bgk(x, 0.55),
          "kbc": lambda x: col.kbc_collide(x, 0.55),
          "reg": lambda x: col.reg_collide(x, 0.55),
          "nco": lambda x: col.nco_collide(x, 0.55, theta)}[op]
    base = fn(f)
    for g in range(48):
        p = L.G_VPERM[g]
        assert np.allclose(fn(f[:, p]), base[:, p], atol=1e-15)


def test_kupershtokh_source_moments():
    """S only touches orders 1 and 2: sqrt3 rho du and 3 rho[(u+du)(u+du) - uu]."""
    f = _random_f(20, 13)
    rng = np.random.default_rng(14)
    F = rng.uniform(-1e-3, 1e-3, size=(20, 3))
    S = col.kupershtokh_source(f, F)
    rho, u = col.macroscopic(f)
    dm = col.moments(S)
    du = F / rho[:, None]
    assert np.allclose(dm[:, 0], 0.0, atol=1e-16)
    assert np.allclose(dm[:, 1:4], np.sqrt(3.0) * rho[:, None] * du, atol=1e-16)
    v = u + du
    exp2 = {"xx": (0, 0), "xy": (0, 1), "xz": (0, 2), "yy": (1, 1), "yz": (1, 2), "zz": (2, 2)}
    for k, name in enumerate(L.MOMENT_NAMES):
        if name in exp2:
            a, b = exp2[name]
            assert np.allclose(dm[:, k], 3.0 * rho * (v[:, a] * v[:, b] - u[:, a] * u[:, b]), atol=1e-16)
        elif L.MOMENT_ORDER[k] >= 3:
            assert np.allclose(dm[:, k], 0.0, atol=1e-15)  # cancellation of two O(1) equilibria


def test_reg_equals_the_latt_chopard_population_formula():
    """Latt & Chopard (2006) in population space: f* = f^eq + (1 - 1/tau) w_i/(2 cs^4)
    Q_i : Pi^neq with Q_i = c_i c_i - cs^2 I and Pi^neq = sum_i c_i c_i (f_i - f^eq_i)."""
    f = _random_f(32, 21)
    tau = 0.58
    rho, u = col.macroscopic(f)
    feq = col.equilibrium(rho, u)
    c = L.C.astype(float)
    cs2 = 1.0 / 3.0
    pi_neq = np.einsum("ia,ib,ni->nab", c, c, f - feq)
    Qi = np.einsum("ia,ib->iab", c, c) - cs2 * np.eye(3)[None]
    fneq2 = L.W[None, :] / (2 * cs2 ** 2) * np.einsum("iab,nab->ni", Qi, pi_neq)
    ref = feq + (1.0 - 1.0 / tau) * fneq2
    assert np.allclose(col.reg_collide(f, tau), ref, atol=1e-15)


def test_reg_removes_higher_order_moments_and_is_bgk_on_second_order_states():
    f = _random_f(32, 22)
    tau = 0.6
    fs = col.reg_collide(f, tau)
    order = np.asarray(L.MOMENT_ORDER)
    assert np.abs(col.moments(fs)[:, order >= 3]).max() < 1e-14 * np.abs(col.moments(f)).max()
    # a state whose non-equilibrium part is purely second order: REG = BGK
    rho, u = col.macroscopic(f)
    g = col.equilibrium(rho, u) + (col.reg_collide(f, 1.0 / 0.7) - col.equilibrium(rho, u))
    assert np.allclose(col.reg_collide(g, tau), col.bgk(g, tau), atol=1e-15)


def test_deep_network_invariance_and_conservation():
    """The 27-20-20-20-4 network (1484 parameters, Sec. IV): the group average is invariant
    under all 48 elements and the collision conserves mass and momentum."""
    sizes = (27, 20, 20, 20, 4)
    theta = lbm_inputs.nco_parameters(3, sizes)
    assert theta.size == 1484
    f = _random_f(8, 31)
    out = col.invariant_network(f, theta, sizes)
    for g in range(48):
        assert np.allclose(col.invariant_network(f[:, L.G_VPERM[g]], theta, sizes), out, atol=1e-13)
    fs = col.nco_collide(f, 0.56, theta, sizes)
    c = L.C.astype(float)
    assert np.allclose(fs.sum(-1), f.sum(-1), rtol=1e-14, atol=0)
    assert np.allclose(fs @ c, f @ c, rtol=0, atol=1e-15)
