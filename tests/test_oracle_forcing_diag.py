"""Pins of oracle.forcing and oracle.diagnostics (CPU only)."""

import math

import numpy as np
import pytest

import lbm_inputs
from oracle import collision as col
from oracle import diagnostics as D
from oracle import forcing as F
from oracle import stepper as S
from oracle import lattice as L


def test_forced_modes_are_the_32_modes_of_the_first_two_shells():
    modes = F.forced_modes(1.0, 2.0)
    assert len(modes) == 16  # half space; with the conjugates 32 modes
    k2 = (modes * modes).sum(axis=1)
    assert sorted(np.bincount(k2).tolist()[1:]) == sorted([3, 6, 4, 3])
    full = {tuple(k) for k in modes} | {tuple(-k) for k in modes}
    assert len(full) == 32


def test_unit_vectors_are_orthonormal_and_normal_to_k():
    for k in F.forced_modes(1.0, 2.0):
        e1, e2 = F.unit_vectors(k)
        assert abs(e1 @ e1 - 1) < 1e-15 and abs(e2 @ e2 - 1) < 1e-15
        assert abs(e1 @ e2) < 1e-15
        assert abs(e1 @ k) < 1e-14 and abs(e2 @ k) < 1e-14


def test_amplitude_integral():
    from scipy.integrate import quad
    val = quad(lambda k: math.exp(-((k - 1.5) ** 2) / 0.5), 1.0, 2.0)[0]
    assert F.amplitude(2.0, 1.5, 0.5, 1.0, 2.0) == pytest.approx(2.0 / val, rel=1e-12)


def test_projection_matches_fft():
    _, u = lbm_inputs.isotropic_field(8, 3, 0.04)
    u = np.moveaxis(u, 0, -1)
    modes = F.forced_modes()
    uh = F.project(u, modes)
    full = np.fft.fftn(u, axes=(0, 1, 2)) / 8 ** 3
    for m, (kx, ky, kz) in enumerate(modes):
        assert np.allclose(uh[m], full[kz % 8, ky % 8, kx % 8], atol=1e-15)


def test_force_is_solenoidal_uncorrelated_and_real():
    _, u = lbm_inputs.isotropic_field(8, 4, 0.04)
    u = np.moveaxis(u, 0, -1)
    modes = F.forced_modes()
    phi, psi = lbm_inputs.forcing_draws(1, seed=5)
    uh = F.project(u, modes)
    fh = F.force_coefficients(uh, phi[0], psi[0], modes, 1e-6, 1.5, 0.5, 1.0, 2.0)
    for m, k in enumerate(modes):
        assert abs(fh[m] @ k) < 1e-18  # k . F^ = 0
        assert abs((np.conj(uh[m]) @ fh[m]).real) < 1e-18  # Re(u^* . F^) = 0
    fx = F.synthesize(fh, modes, (8, 8, 8))
    # F(x) is divergence free spectrally and its projection returns F^
    assert np.allclose(F.project(fx, modes), fh, atol=1e-18)
    # |A_ran|^2 + |B_ran|^2 = F(k)/(2 pi k^2)
    A = F.amplitude(1e-6, 1.5, 0.5, 1.0, 2.0)
    for m, k in enumerate(modes):
        kk = math.sqrt(float(k @ k))
        assert (np.abs(fh[m]) ** 2).sum() == pytest.approx(A * math.exp(-((kk - 1.5) ** 2) / 0.5) / (2 * math.pi * kk * kk), rel=1e-12)


def test_forced_step_injects_momentum_through_source():
    n = 8
    rho, u = lbm_inputs.isotropic_field(n, 6, 0.04)
    u = np.moveaxis(u, 0, -1)
    phi, psi = lbm_inputs.forcing_draws(3, seed=7)
    forcing = F.SpectralForcing(phi, psi, power=1e-5)
    sim = S.Simulation.from_macroscopic(rho, u, 0.52, forcing=forcing)
    f0 = sim.f.copy()
    fstar = sim.post_collision()
    force = F.synthesize(forcing.last_fhat, forcing.modes, (n, n, n))
    c = L.C.astype(float)
    assert np.allclose((fstar - f0) @ c, force, atol=1e-16)
    assert np.allclose(fstar.sum(-1), f0.sum(-1), atol=1e-15)


def test_shell_index_is_nearest_integer():
    k2 = np.arange(0, 200000)
    n = D.shell_index(k2)
    pos = k2 > 0
    assert ((n * n - n + 1 <= k2) & (k2 <= n * n + n))[pos].all()
    ref = np.array([int(math.floor(math.sqrt(v) + 0.5)) for v in k2])
    assert (n == ref).all()


def test_spectrum_parseval_and_single_mode():
    _, u = lbm_inputs.isotropic_field(16, 8, 0.04)
    u = np.moveaxis(u, 0, -1)
    E = D.energy_spectrum(u)
    assert E.sum() == pytest.approx(D.kinetic_energy(u), rel=1e-12)
    # one Fourier mode lands in one bin with energy 1/2 <|u|^2>
    n = 16
    x = lbm_inputs.grid_coordinates(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    for (kx, ky, kz) in [(1, 0, 0), (2, 1, 0), (3, 3, 1), (4, 4, 4)]:
        ph = kx * X + ky * Y + kz * Z
        v = np.stack([np.cos(ph) * 0.01, np.zeros_like(ph), np.zeros_like(ph)], axis=-1)
        E = D.energy_spectrum(v)
        b = int(math.floor(math.sqrt(kx * kx + ky * ky + kz * kz) + 0.5))
        assert E[b] == pytest.approx(D.kinetic_energy(v), rel=1e-12)
        assert np.allclose(np.delete(E, b), 0.0, atol=1e-20)


def test_octant_unfolding_matches_full_field():
    n = 6
    _, uo = lbm_inputs.taylor_green_octant(n, 0.05)
    _, uf = lbm_inputs.taylor_green_3d(2 * n, 0.05, shifted=True)
    un = D.unfold_octant(np.moveaxis(uo, 0, -1))
    assert np.allclose(un, np.moveaxis(uf, 0, -1), atol=1e-15)


def test_dissipation_central_difference_exact_on_quadratic():
    t = np.arange(10) * 0.5
    ke = 3.0 - 0.2 * t + 0.01 * t * t
    d = D.dissipation(ke, 0.5)
    assert np.allclose(d, 0.2 - 0.02 * t[1:-1], atol=1e-13)


def test_spectrum_loss_terms():
    E = np.array([0, 1.0, 2.0, 3.0, 4.0])
    R = np.array([0, 1.0, 1.0, 3.0, 2.0])
    L = D.spectrum_loss(E, R, 2, 4, 20.0, 4)
    assert L == pytest.approx(((1.0) ** 2 + 0 + 1.0) / 3 + 80.0)
