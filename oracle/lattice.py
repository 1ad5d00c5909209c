"""D3Q27 lattice, Hermite moment basis and the O_h symmetry group (FP64).

Test infrastructure only (see the package docstring).

Velocity order (the paper does not fix one): lexicographic over (cz, cy, cx),
each running over (-1, 0, 1); so index 13 is the rest velocity and the
opposite of index i is 26 - i.
"""

import itertools

import numpy as np

# --- Sec. II.A: discrete velocities c_i of the D3Q27 stencil -----------------
C = np.array(
    [(cx, cy, cz) for cz in (-1, 0, 1) for cy in (-1, 0, 1) for cx in (-1, 0, 1)],
    dtype=np.int64,
)  # (27, 3), columns are (x, y, z)
Q = 27

# Sec. II.A names w_i without printing them. The D3Q27 weights are the tensor
# product of the 1-D three-point Gauss-Hermite weights (1/6, 2/3, 1/6).
_W1 = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
W = np.array([_W1[cx] * _W1[cy] * _W1[cz] for cx, cy, cz in C], dtype=np.float64)

CS2 = 1.0 / 3.0  # speed of sound squared, Sec. II.A

OPP = np.array([int(np.where((C == -C[i]).all(axis=1))[0][0]) for i in range(Q)])

# --- Sec. II.B, eq. for M: rows H^(n) in the printed order -----------------
# Each name lists the axis indices a_1..a_n of the Hermite tensor component.
# The last printed row reads "xyxzyz" (garbled); the only sixth-order
# component a D3Q27 stencil can carry is xxyyzz, which is the reading taken.
MOMENT_NAMES = [
    "",
    "x", "y", "z",
    "xx", "xy", "xz", "yy", "yz", "zz",
    "xxy", "xxz", "xyy", "xyz", "xzz", "yyz", "yzz",
    "xxyy", "xxyz", "xxzz", "xyyz", "xyzz", "yyzz",
    "xxyyz", "xxyzz", "xyyzz",
    "xxyyzz",
]
MOMENT_EXPONENTS = np.array(
    [(n.count("x"), n.count("y"), n.count("z")) for n in MOMENT_NAMES], dtype=np.int64
)
MOMENT_ORDER = MOMENT_EXPONENTS.sum(axis=1)


def hermite_1d(n, xi):
    """Probabilists' Hermite polynomial He_n(xi) for n <= 2 (Sec. II.B, eq. H^(n)).

    With the Gaussian weight omega(xi) = (2 pi)^(-1/2) exp(-xi^2/2) the definition
    H^(n) = (-1)^n omega^-1 d^n omega / dxi^n gives 1, xi, xi^2 - 1.
    """
    if n == 0:
        return np.ones_like(xi)
    if n == 1:
        return xi
    if n == 2:
        return xi * xi - 1.0
    raise ValueError("D3Q27 carries at most second order per axis")


def hermite_matrix():
    """The 27x27 moment matrix M of Sec. II.B.

    Row k evaluates the multivariate Hermite component named MOMENT_NAMES[k] at
    the abscissae xi_i = sqrt(3) c_i (Sec. II.B, c_i = xi_i / sqrt(3)). A
    multivariate component with axis counts (e_x, e_y, e_z) is the product of
    the 1-D polynomials He_{e_a}(xi_a), because the Gaussian weight factorises.
    """
    xi = np.sqrt(3.0) * C.astype(np.float64)
    M = np.empty((Q, Q))
    for k, (ex, ey, ez) in enumerate(MOMENT_EXPONENTS):
        M[k] = hermite_1d(ex, xi[:, 0]) * hermite_1d(ey, xi[:, 1]) * hermite_1d(ez, xi[:, 2])
    return M


M = hermite_matrix()
M_INV = np.linalg.inv(M)


# --- Sec. II.B: the octahedral group O_h (48 elements) ---------------------
def group_matrices():
    """All 48 signed 3x3 permutation matrices (rotations and reflections of the cube).

    Enumeration order (ours): axis permutation p in itertools.permutations order,
    then sign vector s in itertools.product((1, -1), repeat=3) order;
    R[a, p[a]] = s[a], i.e. (R c)_a = s_a c_{p(a)}.
    """
    mats = []
    for p in itertools.permutations(range(3)):
        for s in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for a in range(3):
                R[a, p[a]] = s[a]
            mats.append(R)
    return np.array(mats)


G_MATRICES = group_matrices()  # (48, 3, 3)
G = len(G_MATRICES)


def velocity_permutation(R):
    """pi_g with c_{pi_g(i)} = R c_i (Sec. II.B: each g permutes the velocities)."""
    rc = C @ R.T
    perm = np.empty(Q, dtype=np.int64)
    for i in range(Q):
        perm[i] = int(np.where((C == rc[i]).all(axis=1))[0][0])
    return perm


G_VPERM = np.array([velocity_permutation(R) for R in G_MATRICES])  # (48, 27)


def permutation_matrix(perm):
    """Pi_g acting on a population vector: (Pi_g f)_i = f_{pi_g(i)}."""
    P = np.zeros((Q, Q))
    P[np.arange(Q), perm] = 1.0
    return P


def moment_action(g):
    """P_g = M Pi_g M^-1: the action of g on the moment vector (Sec. II.B).

    Returned as a dense FP64 matrix; tests check that it is a signed permutation
    that keeps every moment inside its order.
    """
    return M @ permutation_matrix(G_VPERM[g]) @ M_INV


def moment_action_tables():
    """(perm, sign) integer tables with (P_g m)_k = sign[g,k] * m[perm[g,k]].

    Derived numerically from moment_action and rounded; raises if an entry is
    not a signed permutation.
    """
    perm = np.empty((G, Q), dtype=np.int64)
    sign = np.empty((G, Q), dtype=np.int64)
    for g in range(G):
        P = moment_action(g)
        for k in range(Q):
            row = P[k]
            j = int(np.argmax(np.abs(row)))
            if abs(abs(row[j]) - 1.0) > 1e-12 or np.sum(np.abs(row) > 1e-12) != 1:
                raise AssertionError("moment action is not a signed permutation")
            perm[g, k] = j
            sign[g, k] = int(round(row[j]))
    return perm, sign
