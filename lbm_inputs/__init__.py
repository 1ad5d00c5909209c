"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no lattice Boltzmann arithmetic: it only builds initial
macroscopic fields, network parameters and random draws. Both the oracle and
the CUDA library consume its arrays, so neither depends on the other.

Layout conventions: scalar fields are (nz, ny, nx) arrays; vector fields are
(3, nz, ny, nx) structure-of-arrays (component, z, y, x), float64.
"""

import math

import numpy as np

__all__ = [
    "grid_coordinates", "taylor_green_3d", "taylor_green_2d", "shear_wave",
    "isotropic_field", "nco_parameters", "forcing_draws", "random_populations",
    "NCO_LAYER_SIZES", "reynolds_viscosity",
]

NCO_LAYER_SIZES = (27, 20, 20, 4)


def grid_coordinates(n, length=2.0 * math.pi, shifted=False):
    """Node coordinates x_j = j L/n, or (j + 1/2) L/n when shifted."""
    j = np.arange(n, dtype=np.float64)
    return (j + 0.5 if shifted else j) * (length / n)


def taylor_green_3d(n, u0, shifted=False):
    """rho = 1, u = u0 (sin x cos y cos z, -cos x sin y cos z, 0) on [0, 2 pi)^3.

    shifted=True puts the nodes at (j + 1/2) 2 pi / n, which makes the field
    mirror-symmetric about the planes x, y, z in {0, pi}.
    """
    x = grid_coordinates(n, shifted=shifted)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.stack([
        u0 * np.sin(X) * np.cos(Y) * np.cos(Z),
        -u0 * np.cos(X) * np.sin(Y) * np.cos(Z),
        np.zeros_like(X),
    ])
    return np.ones((n, n, n)), u


def taylor_green_octant(n, u0):
    """The octant [0, pi]^3 of the shifted 3-D Taylor-Green field: n nodes per axis at (j + 1/2) pi / n."""
    rho, u = taylor_green_3d(2 * n, u0, shifted=True)
    return rho[:n, :n, :n].copy(), u[:, :n, :n, :n].copy()


def taylor_green_2d(n, u0, nz=1):
    """z-invariant 2-D Taylor-Green vortex u = u0 (cos x sin y, -sin x cos y, 0)."""
    x = grid_coordinates(n)
    Z, Y, X = np.meshgrid(np.zeros(nz), x, x, indexing="ij")
    u = np.stack([u0 * np.cos(X) * np.sin(Y), -u0 * np.sin(X) * np.cos(Y), np.zeros_like(X)])
    return np.ones((nz, n, n)), u


def shear_wave(n, u0, nz=1, nx=1):
    """u_x = u0 sin(2 pi y / n), one wavelength across the box in y."""
    y = grid_coordinates(n)
    Z, Y, X = np.meshgrid(np.zeros(nz), y, np.zeros(nx), indexing="ij")
    u = np.stack([u0 * np.sin(Y), np.zeros_like(Y), np.zeros_like(Y)])
    return np.ones((nz, n, nx)), u


def isotropic_field(n, seed, u_rms, k_peak=4.0):
    """Random-phase solenoidal velocity with E(k) ~ k^4 exp(-2 (k/k_peak)^2), rho = 1.

    Steps: complex Gaussian modes from default_rng(seed); projection with
    (I - k k^T / k^2); every mode rescaled so that its energy density follows the
    target spectrum divided by the shell area 4 pi k^2; inverse FFT, real part;
    scaled so that u_rms = sqrt(<|u|^2>/3).
    """
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    K = np.stack([KX, KY, KZ])
    k2 = (K * K).sum(axis=0)
    k2s = np.where(k2 == 0, 1.0, k2)
    uh = rng.standard_normal((3, n, n, n)) + 1j * rng.standard_normal((3, n, n, n))
    kdotu = (K * uh).sum(axis=0)
    uh = uh - K * kdotu / k2s
    kk = np.sqrt(k2s)
    target = kk ** 4 * np.exp(-2.0 * (kk / k_peak) ** 2) / (4.0 * math.pi * k2s)
    norm = np.sqrt((np.abs(uh) ** 2).sum(axis=0))
    uh = uh * np.where(norm > 0, np.sqrt(target) / np.where(norm > 0, norm, 1.0), 0.0)
    uh[:, k2 == 0] = 0.0
    u = np.fft.ifftn(uh, axes=(1, 2, 3)).real
    rms = math.sqrt(float((u * u).sum(axis=0).mean()) / 3.0)
    u *= u_rms / rms
    return np.ones((n, n, n)), u


def nco_parameters(seed=0, sizes=NCO_LAYER_SIZES):
    """Kaiming-uniform network parameters as PyTorch's nn.Linear draws them.

    torch.manual_seed(seed), then nn.Linear(27,20), nn.Linear(20,20),
    nn.Linear(20,4) in that order (W ~ U(+-1/sqrt(fan_in)), b likewise).
    Flattened as W1, b1, W2, b2, W3, b3 with every W row-major (out, in).
    Returned as float64 so both consumers read identical numbers.
    """
    import torch

    with torch.random.fork_rng(devices=[]):
        torch.manual_seed(seed)
        layers = [torch.nn.Linear(a, b, dtype=torch.float64) for a, b in zip(sizes[:-1], sizes[1:])]
    parts = []
    for lin in layers:
        parts.append(lin.weight.detach().reshape(-1).numpy())
        parts.append(lin.bias.detach().reshape(-1).numpy())
    return np.concatenate(parts).astype(np.float64)


def forcing_draws(nsteps, nmodes=16, seed=1):
    """Random phases for the spectral force: phi ~ U[0, pi), psi ~ U[0, 2 pi), shape (nsteps, nmodes)."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, math.pi, size=(nsteps, nmodes))
    psi = rng.uniform(0.0, 2.0 * math.pi, size=(nsteps, nmodes))
    return phi, psi


def random_populations(shape, seed, low=0.01, high=0.05):
    """Arbitrary positive populations, (27, nz, ny, nx) float64, uniform in [low, high)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(low, high, size=(27,) + tuple(shape))


def reynolds_viscosity(u0, n, re, length=2.0 * math.pi):
    """nu = U0 N / (L Re) in lattice units with L = 2 pi and N nodes per 2 pi."""
    return u0 * n / (length * re)
