"""Convergence study of Sec. III.B (two-dimensional Taylor-Green vortex, extended without a
gradient along z): the L2 deviation of the velocity and pressure fields from the analytic
solution after one time step falls with the mesh resolution.

Setting (the paper gives none): one period per box, x_j = 2 pi j / N, diffusive scaling
U0 = 0.02 * 16 / N at fixed tau (nu = 0.02), rho = 1 + 3 p with the analytic pressure
p = (U0^2 / 4)(cos 2x + cos 2y), equilibrium start. The analytic solution decays as
exp(-2 nu k^2 t) (velocity) and exp(-4 nu k^2 t) (pressure), k = 2 pi / N in lattice
units. The lattice Boltzmann method is second-order accurate, so the error ratio between
N and 2N must be close to 4.
"""

import numpy as np
import pytest

import lbm_inputs
from oracle import collision as col
from oracle import stepper as S

NU = 0.02


def tgv2d_fields(n):
    u0 = 0.02 * 16 / n
    x = np.arange(n) * 2 * np.pi / n
    Y, X = np.meshgrid(x, x, indexing="ij")
    ux = u0 * np.cos(X) * np.sin(Y)
    uy = -u0 * np.sin(X) * np.cos(Y)
    p = 0.25 * u0 ** 2 * (np.cos(2 * X) + np.cos(2 * Y))
    return ux, uy, p


def l2_errors(n, rho, u):
    """Relative L2 errors of velocity and pressure after one step; rho (1, n, n), u (1, n, n, 3)."""
    ux, uy, p = tgv2d_fields(n)
    k = 2 * np.pi / n
    dv, dp = np.exp(-2 * NU * k * k), np.exp(-4 * NU * k * k)
    ev = np.sqrt(((u[0, ..., 0] - ux * dv) ** 2 + (u[0, ..., 1] - uy * dv) ** 2).sum()
                 / ((ux * dv) ** 2 + (uy * dv) ** 2).sum())
    ep = np.sqrt((((rho[0] - 1) / 3 - p * dp) ** 2).sum() / ((p * dp) ** 2).sum())
    return ev, ep


def oracle_errors(n, op):
    ux, uy, p = tgv2d_fields(n)
    u = np.stack([ux, uy, np.zeros_like(ux)], -1)[None]
    sim = S.Simulation.from_macroscopic((1 + 3 * p)[None], u, col.tau_from_nu(NU), op=op,
                                        theta=lbm_inputs.nco_parameters(0))
    rho, uu = col.macroscopic(sim.step(1).f)
    return l2_errors(n, rho, uu)


@pytest.mark.parametrize("op", ["bgk", "nco"])
def test_tgv2d_one_step_error_converges_at_second_order(op):
    errs = [oracle_errors(n, op) for n in (16, 32, 64)]
    for (ev0, ep0), (ev1, ep1) in zip(errs[:-1], errs[1:]):
        assert np.log2(ev0 / ev1) > 1.9
        assert np.log2(ep0 / ep1) > 1.9
