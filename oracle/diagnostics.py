"""Diagnostics in FP64: kinetic energy, dissipation, energy spectrum, loss (Secs. II.D, III.C, IV, IV.A).

Test infrastructure only (see the package docstring).
Velocity fields are arrays shaped (nz, ny, nx, 3).
"""

import numpy as np


def kinetic_energy(u):
    """k = (1/2) <|u|^2>, the cell average without density weighting.

    Reading of "incompressible kinetic energy" (Sec. IV.A).
    """
    return 0.5 * float((u * u).sum(axis=-1).mean())


def dissipation(ke, dt):
    """-dk/dt by central differences on a uniformly sampled series (Sec. III.C).

    Returns values at the interior samples 1..n-2.
    """
    ke = np.asarray(ke, dtype=np.float64)
    return -(ke[2:] - ke[:-2]) / (2.0 * dt)


DISSIPATION_SAMPLES = 100   # Sec. IV: points of the dissipation curve compared by the loss
DISSIPATION_T_END = 15.0    # Sec. IV: the compared interval is t in [0, 15]


def dissipation_sample_times(t_end=DISSIPATION_T_END, nsamples=DISSIPATION_SAMPLES):
    """The kinetic-energy sampling times of the dissipation loss.

    Sec. IV compares -dk/dt at 100 points between t = 0 and t = 15. Reading: k is sampled
    on the uniform grid t_j = j t_end / (nsamples + 1), j = 0..nsamples+1, and the central
    differences of dissipation() give -dk/dt at the nsamples interior points.
    Returns (times, dt).
    """
    dt = t_end / (nsamples + 1)
    return dt * np.arange(nsamples + 2), dt


def dissipation_mse(ke, dt, eps_ref):
    """L = mean_s (eps_s - eps_ref_s)^2 with eps = -dk/dt from dissipation(ke, dt) (Sec. IV:
    the mean squared error of the dissipation rates against the reference at the sampled
    points). ke holds len(eps_ref) + 2 samples spaced dt apart."""
    eps = dissipation(ke, dt)
    eps_ref = np.asarray(eps_ref, dtype=np.float64)
    if eps.shape != eps_ref.shape:
        raise ValueError(f"{eps.size} dissipation samples against {eps_ref.size} reference values")
    d = eps - eps_ref
    return float((d * d).mean())


def wavenumbers(n):
    """Integer FFT wave numbers 0, 1, ..., n/2-1, -n/2, ..., -1 for a 2 pi box."""
    return np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)


def shell_index(k2):
    """Shell n of an integer |k|^2: the n with n^2 - n + 1 <= |k|^2 <= n^2 + n.

    This is n = round(|k|); |k|^2 is an integer and never equals (n + 1/2)^2,
    so there are no ties. Computed here by direct search in integers.
    """
    k2 = np.asarray(k2, dtype=np.int64)
    n = np.zeros_like(k2)
    # smallest n with n^2 + n >= k2
    while True:
        low = n * n + n < k2
        if not low.any():
            break
        n = n + low
    return n


def energy_spectrum(u, nbins=None):
    """E(n) = sum_{k in shell n} (1/2)|u^(k)|^2 with u^ = FFT(u)/N^3.

    Sec. II.D uses E(kappa) without defining the binning; the shell rule of
    shell_index (nearest integer |k|) is the reading taken.
    """
    nz, ny, nx = u.shape[:3]
    uh = np.fft.fftn(u, axes=(0, 1, 2)) / (nx * ny * nz)
    e = 0.5 * (np.abs(uh) ** 2).sum(axis=-1)
    kz, ky, kx = np.meshgrid(wavenumbers(nz), wavenumbers(ny), wavenumbers(nx), indexing="ij")
    shell = shell_index(kx * kx + ky * ky + kz * kz)
    if nbins is None:
        nbins = int(shell.max()) + 1
    return np.bincount(shell.ravel(), weights=e.ravel(), minlength=nbins)[:nbins]


def unfold_octant(u):
    """Mirror-unfold an octant field (nodes at (j+1/2) dx) to the full (2N)^3 box.

    Taylor-Green parities: u_x is odd in x and even in y and z; u_y is odd in y;
    u_z is odd in z. The octant holds the first N nodes of each axis.
    """
    out = u
    for arr_axis, comp in ((2, 0), (1, 1), (0, 2)):
        mirrored = np.flip(out, axis=arr_axis).copy()
        mirrored[..., comp] *= -1.0
        out = np.concatenate([out, mirrored], axis=arr_axis)
    return out


def spectrum_loss(E, E_ref, kmin, kmax, omega, k_last):
    """L = mean_{kmin<=k<=kmax} ((E - E_ref)/E_ref)^2 + omega E(k_last).

    Sec. II.D combines an MSE between spectra with omega E(kappa_max). Reading
    for the reduced Taylor-Green training: the relative discrepancy is used so
    that every shell counts alike; omega = 20 (Sec. III.A).
    """
    E = np.asarray(E, dtype=np.float64)
    E_ref = np.asarray(E_ref, dtype=np.float64)
    sl = slice(kmin, kmax + 1)
    rel = (E[sl] - E_ref[sl]) / E_ref[sl]
    return float((rel * rel).mean() + omega * E[k_last])
