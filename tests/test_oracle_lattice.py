"""Pins of oracle.lattice against what the paper and the mathematics fix (CPU only)."""

from fractions import Fraction

import numpy as np
import pytest

from oracle import lattice as L
from tests.conftest import read_golden


def test_weights_match_textbook_values():
    rows = [r.split() for r in read_golden("d3q27_weights.txt")]
    c2 = (L.C * L.C).sum(axis=1)
    for sq, count, num, den in rows:
        sel = c2 == int(sq)
        assert sel.sum() == int(count)
        assert np.allclose(L.W[sel], float(Fraction(int(num), int(den))), rtol=0, atol=1e-16)


def test_weight_moments_isotropy():
    c = L.C.astype(float)
    assert abs(L.W.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", L.W, c, c), np.eye(3) / 3.0, atol=1e-15)
    assert abs((L.W * c[:, 0] ** 2 * c[:, 1] ** 2).sum() - 1.0 / 9.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", L.W, c), 0.0, atol=1e-16)


def test_opposite_and_rest_index():
    assert (L.C[13] == 0).all()
    assert (L.C[L.OPP] == -L.C).all()
    assert (L.OPP == 26 - np.arange(27)).all()


def test_hermite_rows_follow_rodrigues_definition():
    """H^(n) = (-1)^n / omega * nabla^n omega, omega the 3-D Gaussian (Sec. II.B)."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    omega = sp.exp(-(x * x + y * y + z * z) / 2)
    xi = np.sqrt(3.0) * L.C.astype(float)
    axes = {"x": x, "y": y, "z": z}
    for k, name in enumerate(L.MOMENT_NAMES):
        expr = omega
        for a in name:
            expr = sp.diff(expr, axes[a])
        poly = sp.simplify((-1) ** len(name) * expr / omega)
        fn = sp.lambdify((x, y, z), poly, "numpy")
        vals = np.broadcast_to(np.asarray(fn(xi[:, 0], xi[:, 1], xi[:, 2]), float), (27,))
        assert np.allclose(L.M[k], vals, atol=1e-12), name


def test_hermite_norms_and_orthogonality():
    rows = dict(r.split() for r in read_golden("hermite_norms.txt"))
    gram = L.M @ np.diag(L.W) @ L.M.T
    names = ["0" if n == "" else n for n in L.MOMENT_NAMES]
    expected = np.array([float(rows[n]) for n in names])
    assert np.allclose(gram, np.diag(expected), atol=1e-13)
    assert np.linalg.matrix_rank(L.M) == 27
    # inverse through the orthogonality identity M^-1 = W M^T N^-1
    assert np.allclose(L.M_INV, np.diag(L.W) @ L.M.T @ np.diag(1.0 / expected), atol=1e-13)


def test_moments_per_order():
    counts = np.bincount(L.MOMENT_ORDER)
    assert counts.tolist() == [1, 3, 6, 7, 6, 3, 1]
    assert (np.diff(L.MOMENT_ORDER) >= 0).all(), "rows are ordered by order"


def test_group_is_the_full_octahedral_group():
    mats = L.G_MATRICES
    assert len(mats) == 48
    keys = {m.tobytes() for m in mats}
    assert len(keys) == 48
    for a in mats:
        assert (a @ a.T == np.eye(3, dtype=int)).all()
        for b in mats:
            assert (a @ b).tobytes() in keys  # closure


def test_velocity_permutations_are_symmetries():
    for g in range(48):
        p = L.G_VPERM[g]
        assert sorted(p.tolist()) == list(range(27))
        assert np.allclose(L.W[p], L.W)
        assert (L.C[p] == L.C @ L.G_MATRICES[g].T).all()


def test_moment_action_is_signed_permutation_within_order():
    perm, sign = L.moment_action_tables()
    for g in range(48):
        assert sorted(perm[g].tolist()) == list(range(27))
        assert (L.MOMENT_ORDER[perm[g]] == L.MOMENT_ORDER).all()
        assert set(np.unique(sign[g]).tolist()) <= {-1, 1}
    # the identity is in the group and maps every moment to itself
    ident = [g for g in range(48) if (L.G_MATRICES[g] == np.eye(3, dtype=int)).all()]
    assert len(ident) == 1
    assert (perm[ident[0]] == np.arange(27)).all() and (sign[ident[0]] == 1).all()


def test_equivariance_commutator_depends_on_rates_per_order():
    """Pi_g M^-1 S M = M^-1 S M Pi_g holds iff S is constant within each order (Sec. II.B)."""
    rng = np.random.default_rng(3)
    s_order = rng.uniform(0.5, 1.9, size=7)
    S = np.diag(s_order[L.MOMENT_ORDER])
    A = L.M_INV @ S @ L.M
    for g in range(48):
        P = L.permutation_matrix(L.G_VPERM[g])
        assert np.allclose(P @ A, A @ P, atol=1e-12)
    # distinct rates inside order 3 break it for some g
    s = s_order[L.MOMENT_ORDER].copy()
    s[10] += 0.3
    A2 = L.M_INV @ np.diag(s) @ L.M
    broken = [g for g in range(48)
              if not np.allclose(L.permutation_matrix(L.G_VPERM[g]) @ A2,
                                 A2 @ L.permutation_matrix(L.G_VPERM[g]), atol=1e-12)]
    assert broken
