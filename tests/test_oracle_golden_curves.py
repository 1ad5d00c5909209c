"""CPU checks of the stored oracle curves (tests/golden/*_ke.txt): they were written by the
oracle from the stated setting, so their first sample must equal the oracle's kinetic
energy of the stated initial field, the samples must be the stated steps, and the energy
must decay over the run (a viscous flow without forcing loses energy; the weakly
compressible solver exchanges a little with acoustic waves, so single samples may rise
slightly)."""

import os

import numpy as np
import pytest

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


GOLDEN_20TC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tgv64_re1600_nco_20tc.txt")


def _rows_20tc():
    ks, es = [], {}
    for ln in open(GOLDEN_20TC):
        if not ln.strip() or ln.startswith("#"):
            continue
        f = ln.split()
        if f[0] == "k":
            ks.append((float(f[1]), float(f[2])))
        else:
            assert f[0] == "E"
            es[int(f[1])] = np.array([float(v) for v in f[2:]])
    return np.array(ks), es


def test_tgv64_20tc_curve_steps_start_and_header():
    """4080 steps = 20.03 convective times N / (2 pi U0); k every 10 steps, E every 1020."""
    g, E = _rows_20tc()
    assert np.array_equal(g[:, 0], np.arange(0, 4081, 10))
    assert sorted(E) == [0, 1020, 2040, 3060, 4080]
    assert 4080 / (64 / (2 * np.pi * 0.05)) > 20.0
    assert abs(g[0, 1] - 0.05 ** 2 / 8) / (0.05 ** 2 / 8) < 1e-6
    nu = lbm_inputs.reynolds_viscosity(0.05, 64, 1600.0)
    assert f"nu = {nu:.17e}" in open(GOLDEN_20TC).read()
    assert g[-1, 1] < 0.2 * g[0, 1]  # most of the energy is dissipated over 20 convective times


def test_tgv64_20tc_curve_continues_the_400_step_curve():
    """Both files are the same oracle run over the same steps: the first 41 samples agree
    with the 400-step curve (the collision is evaluated on slabs there, which changes only
    the rounding order of library matrix products)."""
    g, _ = _rows_20tc()
    g400 = _rows()
    assert np.array_equal(g[:41, 0], g400[:, 0])
    assert np.max(np.abs(g[:41, 1] - g400[:, 1]) / g400[:, 1]) < 1e-12


def test_tgv64_20tc_spectra_sum_to_the_kinetic_energy_and_start_in_one_shell():
    """Parseval: sum_n E(n) = (1/2) <|u|^2> = k at every stored time. The Taylor-Green field
    has all its energy in the modes (+-1, +-1, +-1), |k| = sqrt 3, which the nearest-integer
    shell rule puts in shell 2."""
    g, E = _rows_20tc()
    k = dict(zip(g[:, 0].astype(int), g[:, 1]))
    for t, e in E.items():
        assert len(e) == 56  # shells 0 .. round(sqrt(3) * 32)
        assert abs(e.sum() - k[t]) / k[t] < 1e-12, t
        assert np.all(e >= 0.0)
    e0 = E[0]
    assert abs(e0[2] - k[0]) / k[0] < 1e-12
    assert np.sum(np.delete(e0, 2)) < 1e-12 * k[0]
    # energy moves to higher shells as the vortex breaks down
    assert E[4080][8:].sum() / E[4080].sum() > E[1020][8:].sum() / E[1020].sum()


def _rows_hit(op):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"hit64_forced_{op}.txt")
    if not os.path.exists(path):
        pytest.skip(f"{os.path.basename(path)} has not been written (tests/golden/make_hit64_forced.py {op})")
    header, ks, es = "", [], {}
    for ln in open(path):
        if ln.startswith("#"):
            header += ln
            continue
        f = ln.split()
        if f[0] == "k":
            ks.append((float(f[1]), float(f[2])))
        else:
            assert f[0] == "E"
            es[int(f[1])] = np.array([float(v) for v in f[2:]])
    return header, np.array(ks), es


def test_forced_hit64_curves_steps_start_and_parseval():
    """The stored forced runs (BGK and NCO): k every 10 steps and spectra every 100 steps over
    1000 steps; both start at the oracle's k of the FP32-rounded seed-1 field; the header's
    power is nu <|grad u|^2> of that field; Parseval (sum_n E(n) = k) at every stored time;
    the force keeps k of the order of its start."""
    rho, u = lbm_inputs.isotropic_field(64, 1, 0.04)
    u32 = u.astype(np.float32).astype(np.float64)
    f0 = col.equilibrium(rho.astype(np.float32).astype(np.float64), np.moveaxis(u32, 0, -1))
    _, u0 = col.macroscopic(f0)
    grads = [np.gradient(u32[a], axis=ax) for a in range(3) for ax in range(3)]
    power = float(0.0015 * np.mean(sum(g * g for g in grads)))
    first = {}
    for op in ("bgk", "nco"):
        header, g, E = _rows_hit(op)
        assert np.array_equal(g[:, 0], np.arange(0, 1001, 10))
        assert sorted(E) == list(range(0, 1001, 100))
        assert g[0, 1] == D.kinetic_energy(u0)
        assert f"power = {power!r}" in header
        k = dict(zip(g[:, 0].astype(int), g[:, 1]))
        for t, e in E.items():
            assert np.all(e >= 0.0)
            assert abs(e.sum() - k[t]) / k[t] < 1e-12, (op, t)
        assert 0.5 < g[-1, 1] / g[0, 1] < 2.0
        first[op] = (g, E)
    # the same start, then two different operators
    assert np.array_equal(first["bgk"][1][0], first["nco"][1][0])
    assert abs(first["bgk"][0][-1, 1] - first["nco"][0][-1, 1]) > 1e-6 * first["bgk"][0][-1, 1]
