"""CPU checks of the stored oracle curves (tests/golden/*_ke.txt): they were written by the
oracle from the stated setting, so their first sample must equal the oracle's kinetic
energy of the stated initial field, the samples must be the stated steps, and the energy
must decay over the run (a viscous flow without forcing loses energy; the weakly
compressible solver exchanges a little with acoustic waves, so single samples may rise
slightly)."""

import os

import numpy as np

import lbm_inputs
from oracle import collision as col
from oracle import diagnostics as D

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tgv64_re1600_nco_ke.txt")


def _rows():
    return np.array([[float(a), float(b)] for a, b in
                     (ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#"))])


def test_tgv64_curve_starts_at_the_oracle_kinetic_energy_of_the_fp32_rounded_field():
    rho, u = lbm_inputs.taylor_green_3d(64, 0.05)
    f0 = col.equilibrium(rho.astype(np.float32).astype(np.float64),
                         np.moveaxis(u.astype(np.float32).astype(np.float64), 0, -1))
    _, u0 = col.macroscopic(f0)
    g = _rows()
    assert g[0, 0] == 0
    assert g[0, 1] == D.kinetic_energy(u0)
    # analytic value of the continuous field: k = U0^2 / 8
    assert abs(g[0, 1] - 0.05 ** 2 / 8) / (0.05 ** 2 / 8) < 1e-6


def test_tgv64_curve_samples_and_decay():
    g = _rows()
    assert np.array_equal(g[:, 0], np.arange(0, 401, 10))
    assert g[-1, 1] < g[0, 1]
    assert np.max(np.abs(np.diff(g[:, 1]))) < 1e-2 * g[0, 1]
    header = open(GOLDEN).read()
    nu = lbm_inputs.reynolds_viscosity(0.05, 64, 1600.0)
    assert f"nu = {nu:.17e}" in header
