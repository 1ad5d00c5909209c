"""Collision operators of arXiv 2412.08229 in FP64 (Sec. II.A-B).

Test infrastructure only (see the package docstring).

All functions act on populations shaped (..., 27) in the velocity order of
oracle.lattice. Nothing is fused or reordered beyond what the equations state.
"""

import numpy as np

from .lattice import C, CS2, G, G_VPERM, M, M_INV, MOMENT_ORDER, W

# ---------------------------------------------------------------------------
# Sec. II.A
# ---------------------------------------------------------------------------


def macroscopic(f):
    """rho = sum_i f_i, rho u = sum_i c_i f_i (Sec. II.A, eq. for rho and rho u)."""
    rho = f.sum(axis=-1)
    j = f @ C.astype(np.float64)
    return rho, j / rho[..., None]


def equilibrium(rho, u):
    """Quadratic equilibrium f^eq_i(rho, u) (Sec. II.A, Eq. EquilibriumDistribution)."""
    cu = u @ C.T.astype(np.float64)
    usq = (u * u).sum(axis=-1)
    return W * rho[..., None] * (
        1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq[..., None] / (2.0 * CS2)
    )


def tau_from_nu(nu):
    """nu = c_s^2 (tau - dt/2) with dt = 1 (Sec. II.B, below eq. omegatheta)."""
    return nu / CS2 + 0.5


def bgk(f, tau):
    """BGK: f* = f - (f - f^eq)/tau (Sec. II.A, eq. for Omega_i)."""
    rho, u = macroscopic(f)
    return f - (f - equilibrium(rho, u)) / tau


# ---------------------------------------------------------------------------
# Sec. II.B: the neural collision operator
# ---------------------------------------------------------------------------


def moments(f):
    """m = M f (Sec. II.B)."""
    return f @ M.T


def equilibrium_moments(rho, u):
    """m^eq = M f^eq (Sec. II.B, text below eq. omegatheta)."""
    return moments(equilibrium(rho, u))


def relaxation_diagonal(tau, rates):
    """Diagonal of S_theta = diag(1_{dim+1}, omega_nu, omega_n^NN) (Sec. II.B).

    Orders 0 and 1 (rho, u) relax with rate 1; every second-order moment with
    omega_nu = 1/tau (reading: one rate for the whole second order, which is the
    only reading under which "all rates = 1/tau" is BGK); order 3, 4, 5, 6 with
    rates[..., 0..3] respectively (reading: network outputs in ascending order).
    ``rates`` has shape (..., 4); the result has shape (..., 27).
    """
    rates = np.asarray(rates, dtype=np.float64)
    s = np.empty(rates.shape[:-1] + (27,))
    for k in range(27):
        n = MOMENT_ORDER[k]
        if n <= 1:
            s[..., k] = 1.0
        elif n == 2:
            s[..., k] = 1.0 / tau
        else:
            s[..., k] = rates[..., n - 3]
    return s


def mrt_collide(f, tau, rates):
    """Omega(f) = -M^-1 S_theta (M f - m^eq); returns f + Omega (Sec. II.B, eq. omegatheta)."""
    rho, u = macroscopic(f)
    dm = moments(f) - equilibrium_moments(rho, u)
    s = relaxation_diagonal(tau, rates)
    return f - (s * dm) @ M_INV.T


# --- the invariant network ---------------------------------------------------

LAYER_SIZES = (27, 20, 20, 4)  # Sec. II.B: two hidden layers of 20, 1064 parameters


def unpack_theta(theta, sizes=LAYER_SIZES):
    """Split a flat parameter vector into [(W, b), ...] (PyTorch nn.Linear layout:
    W has shape (out, in), stored row-major, followed by b)."""
    theta = np.asarray(theta, dtype=np.float64)
    layers, off = [], 0
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        Wl = theta[off: off + n_in * n_out].reshape(n_out, n_in)
        off += n_in * n_out
        bl = theta[off: off + n_out]
        off += n_out
        layers.append((Wl, bl))
    if off != theta.size:
        raise ValueError(f"theta has {theta.size} entries, layout needs {off}")
    return layers


def phi_network(x, layers, operand_round=None):
    """The plain network Phi: Linear, ReLU, Linear, ReLU, ..., Linear (Sec. II.B, III).

    operand_round (default None: exact FP64) models a reduced-precision evaluation of the
    hidden layers: when given, it is applied to the input, weights and bias of every layer
    but the output layer, and to every hidden activation that enters such a layer; the
    output layer and its input stay exact. Products and sums are FP64 either way.
    """
    rnd = (lambda a: a) if operand_round is None else operand_round
    h = x
    last = len(layers) - 1
    for li, (Wl, bl) in enumerate(layers):
        if li < last:
            h = rnd(h) @ rnd(Wl).T + rnd(bl)
            h = np.maximum(h, 0.0)
        else:
            h = h @ Wl.T + bl
    return h


def group_moments(f, g):
    """m^(g) = M Pi_g f with (Pi_g f)_i = f_{pi_g(i)} (Sec. II.B)."""
    return moments(f[..., G_VPERM[g]])


def invariant_network(f, theta, sizes=LAYER_SIZES, chunk=8192, operand_round=None):
    """N_Phi(f) = (1/|G|) sum_g Phi(m^(g)) over all 48 g of O_h (Sec. II.B, eq. gconv_m).

    Input: the full raw 27-moment vector of each transformed population set
    (reading: not normalised by rho and not m - m^eq; the 1064-parameter count
    only fits 27 inputs). Evaluated as 48 explicit copies, as the equation reads;
    cells are processed in chunks only to bound memory. operand_round: see phi_network.
    """
    layers = unpack_theta(theta, sizes)
    lead = f.shape[:-1]
    flat = f.reshape(-1, f.shape[-1])
    out = np.empty((flat.shape[0], sizes[-1]))
    for a in range(0, flat.shape[0], chunk):
        fc = flat[a: a + chunk]
        fg = np.take(fc, G_VPERM.ravel(), axis=1).reshape(-1, fc.shape[-1])  # rows (cell, g): Pi_g f
        phi = phi_network(moments(fg), layers, operand_round)  # Phi(m^(g)), m^(g) = M Pi_g f
        out[a: a + chunk] = phi.reshape(fc.shape[0], G, -1).sum(axis=1) / G
    return out.reshape(lead + (sizes[-1],))


def tau_from_network(tau_tilde):
    """tau_n = 1 / (2 (1 + exp(tau~_n))) + 1/2 (Sec. II.B, sigmoid eq.)."""
    return 1.0 / (2.0 * (1.0 + np.exp(tau_tilde))) + 0.5


def nco_rates(f, theta, sizes=LAYER_SIZES, operand_round=None):
    """omega_n = 1/tau_n for the order groups n = 3..6 (Sec. II.B). operand_round: see phi_network."""
    return 1.0 / tau_from_network(invariant_network(f, theta, sizes, operand_round=operand_round))


def nco_collide(f, tau, theta, sizes=LAYER_SIZES):
    """Post-collision populations of the NCO: f + Omega(f, theta) (Sec. II.B, eq. omegatheta)."""
    return mrt_collide(f, tau, nco_rates(f, theta, sizes))


# ---------------------------------------------------------------------------
# REG (compared in Sec. III.A and Sec. IV, cites Latt & Chopard 2006; not defined in the paper)
# ---------------------------------------------------------------------------


def reg_collide(f, tau):
    """Regularised BGK, restated from Latt and Chopard (2006).

    Reading (the paper only names it): the non-equilibrium part is replaced by its
    second-order Hermite projection before relaxing, f* = f^eq + (1 - 1/tau) f^neq_(2).
    In the moment basis of Sec. II.B that is the generalised relaxation with every
    moment of order 3..6 relaxed with rate 1 (the equilibrium has none), so
    S = diag(1, 1, 1/tau, 1, 1, 1, 1) over the orders 0..6.
    """
    return mrt_collide(f, tau, np.ones(np.shape(f)[:-1] + (4,)))


# ---------------------------------------------------------------------------
# KBC (Sec. III cites Karlin, Boesch & Chikatamarla 2014; not defined in the paper)
# ---------------------------------------------------------------------------


def kbc_collide(f, tau, gamma_override=None):
    """Entropic KBC collision, restated from Karlin, Boesch and Chikatamarla (2014).

    Reading (the paper only cites it): split the non-equilibrium part in the
    Hermite basis into Delta s = all second-order moments and Delta h = orders
    3..6, both mapped back with M^-1; beta = 1/(2 tau);
    gamma = 1/beta - (2 - 1/beta) <Ds|Dh>/<Dh|Dh> with <X|Y> = sum X_i Y_i / f^eq_i;
    f* = f - beta (2 Ds + gamma Dh). If <Dh|Dh> < 1e-30, gamma = 2 (BGK).
    """
    rho, u = macroscopic(f)
    feq = equilibrium(rho, u)
    dm = moments(f) - moments(feq)
    ds_m = np.where(MOMENT_ORDER == 2, dm, 0.0)
    dh_m = np.where(MOMENT_ORDER >= 3, dm, 0.0)
    ds = ds_m @ M_INV.T
    dh = dh_m @ M_INV.T
    beta = 1.0 / (2.0 * tau)
    if gamma_override is not None:
        gamma = np.full(rho.shape, float(gamma_override))
    else:
        sh = (ds * dh / feq).sum(axis=-1)
        hh = (dh * dh / feq).sum(axis=-1)
        safe = hh >= 1e-30
        gamma = np.where(
            safe, 1.0 / beta - (2.0 - 1.0 / beta) * sh / np.where(safe, hh, 1.0), 2.0
        )
    return f - beta * (2.0 * ds + gamma[..., None] * dh)


# ---------------------------------------------------------------------------
# Kupershtokh exact-difference forcing (Sec. II.A)
# ---------------------------------------------------------------------------


def kupershtokh_source(f, force):
    """S_i = f^eq(rho, u + du) - f^eq(rho, u), du = F dt / rho (Sec. II.A).

    Reading: u in both equilibria is the bare u = j / rho of the pre-collision
    populations; dt = 1. ``force`` has shape (..., 3).
    """
    rho, u = macroscopic(f)
    du = force / rho[..., None]
    return equilibrium(rho, u + du) - equilibrium(rho, u)
