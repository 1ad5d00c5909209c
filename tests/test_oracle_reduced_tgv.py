"""The reduced Taylor-Green domain of Appendix A, [0, pi/2]^3 (1/64 of the periodic box):
its symmetry boundary conditions, derived here from the flow's symmetry group, must give
exactly the restriction of the full periodic simulation (the paper's own check at the end
of Appendix A), for any collision operator that respects the cube symmetries."""

import numpy as np
import pytest

import lbm_inputs
from oracle import collision as col
from oracle import stepper as S


def test_tgv_symmetry_group_tiles_the_box_with_the_reduced_domain():
    group = S.tgv_symmetry_group()
    assert len(group) == 64
    rng = np.random.default_rng(1)
    pts = rng.uniform(0.0, np.pi / 2, (500, 3))
    blocks = set()
    for A, k in group:
        img = (pts @ A.T + k * np.pi / 2) % (2 * np.pi)
        b = {tuple(v) for v in np.floor(img / (np.pi / 2)).astype(int)}
        assert len(b) == 1      # the domain maps onto one block
        blocks |= b
    assert len(blocks) == 64    # and the 64 images tile the box once


@pytest.mark.parametrize("op", ["bgk", "nco"])
def test_reduced_domain_equals_the_full_box_restriction(op):
    n = 4                       # reduced: 4^3 nodes; full periodic box: 16^3 nodes
    nu = 0.01
    theta = lbm_inputs.nco_parameters(0)
    rho, u = lbm_inputs.taylor_green_3d(4 * n, 0.05, shifted=True)
    full = S.Simulation.from_macroscopic(rho, np.moveaxis(u, 0, -1), col.tau_from_nu(nu), op=op, theta=theta)
    red = S.Simulation.from_macroscopic(rho[:n, :n, :n], np.moveaxis(u[:, :n, :n, :n], 0, -1),
                                        col.tau_from_nu(nu), op=op, theta=theta, bc="tgv_reduced")
    full.step(3)
    red.step(3)
    assert np.abs(red.f - full.f[:n, :n, :n]).max() <= 1e-14


def test_library_reduced_table_matches_the_oracle_group_bit_exactly():
    """The CUDA library derives its own table in C++ (host code, no GPU needed); for every
    block around the domain the symmetry it picks must be the oracle's, and its direction
    map must send c_i to A c_i."""
    P = pytest.importorskip("paper_2412_08229_gb300")
    from oracle import lattice as L
    A_lib, k_lib, pm_lib = P.lbm_tgv_reduced_table()
    group = S.tgv_symmetry_group()
    for r in range(27):
        if r == 13:
            continue
        centre = np.array([r % 3 - 1, (r // 3) % 3 - 1, r // 9 - 1]) + 0.5
        hits = [(A, k) for A, k in group if (((A @ centre + k) % 4 > 0) & ((A @ centre + k) % 4 < 1)).all()]
        assert len(hits) == 1
        A, k = hits[0]
        assert np.array_equal(A_lib[r], A) and np.array_equal(k_lib[r], k)
        for i in range(27):
            assert np.array_equal(L.C[pm_lib[r, i]], A @ L.C[i])
