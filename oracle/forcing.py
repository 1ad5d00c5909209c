"""Alvelius spectral forcing in FP64 (Sec. II.C).

Test infrastructure only (see the package docstring).

Grid coordinates are x_j = 2 pi j / N on the periodic box [0, 2 pi)^3, wave
vectors k are integer triples, and Fourier coefficients are normalised as
    u^(k) = N^-3 sum_x u(x) exp(-i k.x),      u(x) = sum_k u^(k) exp(i k.x).

Readings taken where Sec. II.C is silent or garbled:
  * forced modes: integer k with ka <= |k| <= kb; only the half space
    (kz > 0, or kz = 0 and ky > 0, or kz = ky = 0 and kx > 0) is drawn, the
    other half is its complex conjugate, so F(x) = sum_half 2 Re(F^(k) e^{ik.x});
  * e1 is printed as (kx ky, -kx ky, 0)/sqrt(kx^2+ky^2), which is not normal to
    k; Alvelius' e1 = (ky, -kx, 0)/sqrt(kx^2+ky^2) is used. For kx = ky = 0,
    e1 = (1, 0, 0) and e2 = (0, 1, 0);
  * the leading "e" before tan(theta_1) is a typo; theta_1 = atan2(num, den);
  * dt = 1; the integral defining A is the continuous Gaussian over [ka, kb];
  * the velocity projected is the bare u = j/rho of the pre-collision state,
    lagged by one step (step n uses the projection made during step n-1; step 0
    uses the initial field).
"""

import math

import numpy as np


def forced_modes(ka=1.0, kb=2.0):
    """Half-space integer wave vectors with ka <= |k| <= kb, sorted by (|k|^2, kz, ky, kx)."""
    r = int(math.floor(kb))
    modes = []
    for kz in range(-r, r + 1):
        for ky in range(-r, r + 1):
            for kx in range(-r, r + 1):
                k2 = kx * kx + ky * ky + kz * kz
                if not (ka * ka <= k2 <= kb * kb):
                    continue
                if kz > 0 or (kz == 0 and ky > 0) or (kz == 0 and ky == 0 and kx > 0):
                    modes.append((kx, ky, kz))
    modes.sort(key=lambda k: (k[0] ** 2 + k[1] ** 2 + k[2] ** 2, k[2], k[1], k[0]))
    return np.array(modes, dtype=np.int64)


def unit_vectors(k):
    """e1, e2 normal to k and to each other (Sec. II.C, eqs. for e_1 and e_2)."""
    kx, ky, kz = (float(v) for v in k)
    kk = math.sqrt(kx * kx + ky * ky + kz * kz)
    kh = math.sqrt(kx * kx + ky * ky)
    if kh == 0.0:
        return np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    e1 = np.array([ky, -kx, 0.0]) / kh
    e2 = np.array([kx * kz / kk, ky * kz / kk, -kh * kh / kk]) / kh
    return e1, e2


def amplitude(power, kf, c, ka, kb):
    """A = (P/dt) / int_ka^kb exp(-(k-kf)^2/c) dk, dt = 1 (Sec. II.C, eq. for A)."""
    integral = 0.5 * math.sqrt(math.pi * c) * (
        math.erf((kb - kf) / math.sqrt(c)) - math.erf((ka - kf) / math.sqrt(c))
    )
    return power / integral


def project(u, modes):
    """u^(k) = N^-3 sum_x u(x) e^{-ik.x} on the given modes; u: (nz,ny,nx,3) -> (nmodes,3) complex."""
    nz, ny, nx = u.shape[:3]
    jz, jy, jx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.empty((len(modes), 3), dtype=np.complex128)
    for m, (kx, ky, kz) in enumerate(modes):
        phase = np.exp(-2j * np.pi * (kx * jx / nx + ky * jy / ny + kz * jz / nz))
        for a in range(3):
            out[m, a] = (u[..., a] * phase).sum() / (nx * ny * nz)
    return out


def force_coefficients(uhat, phi, psi, modes, power, kf, c, ka, kb):
    """F^(k) = A_ran e1 + B_ran e2 for every forced half-space mode (Sec. II.C).

    A_ran = (F(k)/(2 pi k^2))^(1/2) e^{i theta1} g_A(phi),
    B_ran = (F(k)/(2 pi k^2))^(1/2) e^{i theta2} g_B(phi),
    F(k) = A exp(-(k-kf)^2/c), g_A = sin 2phi, g_B = cos 2phi,
    theta2 = theta1 + psi, tan theta1 from the printed ratio with xi_i = u^.e_i.
    """
    A = amplitude(power, kf, c, ka, kb)
    out = np.empty((len(modes), 3), dtype=np.complex128)
    for m, k in enumerate(modes):
        kk = math.sqrt(float((k * k).sum()))
        e1, e2 = unit_vectors(k)
        xi1 = complex(np.dot(uhat[m], e1))
        xi2 = complex(np.dot(uhat[m], e2))
        gA = math.sin(2.0 * phi[m])
        gB = math.cos(2.0 * phi[m])
        sp, cp = math.sin(psi[m]), math.cos(psi[m])
        num = gA * xi1.real + gB * (sp * xi2.imag + cp * xi2.real)
        den = -gA * xi1.imag + gB * (sp * xi2.real - cp * xi2.imag)
        theta1 = math.atan2(num, den)
        theta2 = theta1 + psi[m]
        Fk = A * math.exp(-((kk - kf) ** 2) / c)
        amp = math.sqrt(Fk / (2.0 * math.pi * kk * kk))
        a_ran = amp * complex(math.cos(theta1), math.sin(theta1)) * gA
        b_ran = amp * complex(math.cos(theta2), math.sin(theta2)) * gB
        out[m] = a_ran * e1 + b_ran * e2
    return out


def synthesize(fhat, modes, shape):
    """F(x) = sum_half 2 Re(F^(k) e^{ik.x}) on the grid; returns (nz,ny,nx,3)."""
    nz, ny, nx = shape
    jz, jy, jx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.zeros((nz, ny, nx, 3))
    for m, (kx, ky, kz) in enumerate(modes):
        phase = np.exp(2j * np.pi * (kx * jx / nx + ky * jy / ny + kz * jz / nz))
        for a in range(3):
            out[..., a] += 2.0 * (fhat[m, a] * phase).real
    return out


class SpectralForcing:
    """Per-step Alvelius force with externally supplied random draws.

    phi: (nsteps, nmodes) in [0, pi); psi: (nsteps, nmodes) in [0, 2 pi).
    """

    def __init__(self, phi, psi, power, kf=1.5, c=0.5, ka=1.0, kb=2.0):
        self.modes = forced_modes(ka, kb)
        self.phi = np.asarray(phi, dtype=np.float64)
        self.psi = np.asarray(psi, dtype=np.float64)
        if self.phi.shape[1] != len(self.modes) or self.psi.shape != self.phi.shape:
            raise ValueError("draws must have shape (nsteps, nmodes)")
        self.params = dict(power=power, kf=kf, c=c, ka=ka, kb=kb)
        self.uhat_prev = None
        self.last_fhat = None

    def observe(self, u):
        self.uhat_prev = project(u, self.modes)

    def coefficients(self, t):
        return force_coefficients(self.uhat_prev, self.phi[t], self.psi[t], self.modes, **self.params)

    def force_field(self, t, shape):
        self.last_fhat = self.coefficients(t)
        return synthesize(self.last_fhat, self.modes, shape)


class RecordedForcing:
    """A forcing that replays given force fields, one per step, and records nothing.

    Reading for differentiating through forced steps: the spectral force of a step is an
    input of that step (the stirring is redrawn every step and its phase is chosen to be
    uncorrelated with the flow), so gradients do not flow through its dependence on the
    velocity. ``fields[t]`` has shape (nz, ny, nx, 3). ``wrap`` records the fields an
    existing forcing produces, for a replay with the same forces.
    """

    def __init__(self, fields=None, wrap=None):
        self.fields = [] if fields is None else [np.asarray(f, dtype=np.float64) for f in fields]
        self.wrap = wrap

    def observe(self, u):
        if self.wrap is not None:
            self.wrap.observe(u)

    def force_field(self, t, shape):
        if self.wrap is not None:
            f = self.wrap.force_field(t, shape)
            self.fields.append(np.array(f, dtype=np.float64))
            return f
        return self.fields[t]
