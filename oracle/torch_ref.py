"""The oracle's step restated in PyTorch CPU float64, differentiable by autograd.

Test infrastructure only (see the package docstring). This is the second, independent
reference for the gradient of a loss through an unrolled simulation: the same equations
as oracle.collision / oracle.stepper (Sec. II.A-B, Appendix A), written with torch ops
so that autograd supplies d loss / d theta. It is itself pinned by central finite
differences of the NumPy oracle (tests/test_oracle_adjoint.py).

Populations are (nz, ny, nx, 27) float64 tensors; theta is the flat parameter vector of
the layer sizes given (1064 for 27-20-20-4, 1484 for 27-20-20-20-4).
"""

import numpy as np
import torch

from . import lattice as L

_C = torch.tensor(L.C, dtype=torch.float64)
_W = torch.tensor(L.W, dtype=torch.float64)
_M = torch.tensor(L.M, dtype=torch.float64)
_MINV = torch.tensor(L.M_INV, dtype=torch.float64)
_ORDER = torch.tensor(L.MOMENT_ORDER)
_VPERM = torch.tensor(L.G_VPERM)
_CS2 = L.CS2


def equilibrium(rho, u):
    """Sec. II.A, Eq. EquilibriumDistribution."""
    cu = u @ _C.T
    usq = (u * u).sum(-1, keepdim=True)
    return _W * rho[..., None] * (1 + cu / _CS2 + cu * cu / (2 * _CS2 ** 2) - usq / (2 * _CS2))


def network(m_g, theta, sizes=(27, 20, 20, 4)):
    """Phi applied to the last axis (Sec. II.B): Linear-ReLU-Linear-ReLU-Linear."""
    h, off = m_g, 0
    n_layers = len(sizes) - 1
    for li, (a, b) in enumerate(zip(sizes[:-1], sizes[1:])):
        Wl = theta[off: off + a * b].reshape(b, a)
        off += a * b
        bl = theta[off: off + b]
        off += b
        h = h @ Wl.T + bl
        if li < n_layers - 1:
            h = torch.relu(h)
    return h


def nco_collide(f, tau, theta, sizes=(27, 20, 20, 4)):
    """f + Omega(f, theta) with the group-averaged network (Sec. II.B, eqs. omegatheta, gconv_m)."""
    rho = f.sum(-1)
    u = (f @ _C) / rho[..., None]
    m = f @ _M.T
    meq = equilibrium(rho, u) @ _M.T
    m_g = f[..., _VPERM] @ _M.T                    # (..., 48, 27)
    tau_tilde = network(m_g, theta, sizes).mean(dim=-2)    # (..., 4)
    tau_n = 1.0 / (2.0 * (1.0 + torch.exp(tau_tilde))) + 0.5
    rates = 1.0 / tau_n
    s = torch.ones(f.shape[:-1] + (27,), dtype=torch.float64)
    s = torch.where(_ORDER == 2, torch.full_like(s, 1.0 / tau), s)
    for n in range(3, 7):
        s = torch.where(_ORDER == n, rates[..., n - 3: n - 2].expand_as(s), s)
    return f - (s * (m - meq)) @ _MINV.T


def stream_periodic(fs):
    out = []
    for i in range(27):
        cx, cy, cz = (int(v) for v in L.C[i])
        out.append(torch.roll(fs[..., i], shifts=(cz, cy, cx), dims=(0, 1, 2)))
    return torch.stack(out, dim=-1)


def stream_mirror(fs):
    """Specular reflection at all faces (the oracle's mirror-octant reading)."""
    from .stepper import reflect_index
    p = fs
    for arr_axis, comp in ((2, 0), (1, 1), (0, 2)):
        refl = torch.tensor(reflect_index(comp))
        lo = p.narrow(arr_axis, 0, 1)[..., refl]
        hi = p.narrow(arr_axis, p.shape[arr_axis] - 1, 1)[..., refl]
        p = torch.cat([lo, p, hi], dim=arr_axis)
    nz, ny, nx = fs.shape[:3]
    out = []
    for i in range(27):
        cx, cy, cz = (int(v) for v in L.C[i])
        out.append(p[1 - cz: 1 - cz + nz, 1 - cy: 1 - cy + ny, 1 - cx: 1 - cx + nx, i])
    return torch.stack(out, dim=-1)


def tgv_reduced_gather(n):
    """Flat source index of every (z, y, x, i) after streaming on the reduced Taylor-Green
    domain (Appendix A): the NumPy oracle's stream_tgv_reduced applied to the array of flat
    indices. Streaming is a permutation, so gathering with it is the same map."""
    from .stepper import stream_tgv_reduced
    ident = np.arange(n * n * n * 27, dtype=np.float64).reshape(n, n, n, 27)
    return torch.tensor(stream_tgv_reduced(ident).astype(np.int64))


def stream(fs, bc, gather=None):
    if bc == "periodic":
        return stream_periodic(fs)
    if bc == "mirror":
        return stream_mirror(fs)
    if bc == "tgv_reduced":
        g = tgv_reduced_gather(fs.shape[0]) if gather is None else gather
        return fs.reshape(-1)[g.reshape(-1)].reshape(fs.shape)
    raise ValueError(bc)


def kupershtokh_source(f, force):
    """S_i = f^eq(rho, u + F / rho) - f^eq(rho, u) with the bare u = j / rho (Sec. II.A)."""
    rho = f.sum(-1)
    u = (f @ _C) / rho[..., None]
    return equilibrium(rho, u + force / rho[..., None]) - equilibrium(rho, u)


def run(f0, tau, theta, nsteps, bc="periodic", sizes=(27, 20, 20, 4), forces=None):
    """Unrolled NCO simulation; returns the pre-collision state after nsteps. ``forces``:
    one (nz, ny, nx, 3) force field per step, taken as given (no gradient through them)."""
    f = f0
    gather = tgv_reduced_gather(f0.shape[0]) if bc == "tgv_reduced" else None
    for t in range(nsteps):
        fs = nco_collide(f, tau, theta, sizes)
        if forces is not None:
            fs = fs + kupershtokh_source(f, torch.as_tensor(forces[t], dtype=torch.float64))
        f = stream(fs, bc, gather)
    return f


def kinetic_energy(f):
    """k = (1/2) <|u|^2> over the cells (the oracle.diagnostics reading of Sec. IV.A)."""
    u = velocity(f)
    return 0.5 * (u * u).sum(-1).mean()


def run_kinetic_energy(f0, tau, theta, obs_steps, bc="periodic", sizes=(27, 20, 20, 4)):
    """k after each of the (increasing) step counts obs_steps of an unrolled NCO run."""
    f = f0
    gather = tgv_reduced_gather(f0.shape[0]) if bc == "tgv_reduced" else None
    out, t = [], 0
    for s in obs_steps:
        while t < s:
            f = stream(nco_collide(f, tau, theta, sizes), bc, gather)
            t += 1
        out.append(kinetic_energy(f))
    return torch.stack(out)


def dissipation_mse(ke, dt, eps_ref):
    """mean_s (-dk/dt - eps_ref)^2 with central differences (oracle.diagnostics, Sec. IV)."""
    eps = -(ke[2:] - ke[:-2]) / (2.0 * dt)
    d = eps - eps_ref
    return (d * d).mean()


def velocity(f):
    return (f @ _C) / f.sum(-1)[..., None]


def unfold_octant(u):
    """Mirror-unfold an octant velocity field (Taylor-Green parities), torch version."""
    out = u
    for arr_axis, comp in ((2, 0), (1, 1), (0, 2)):
        mirrored = torch.flip(out, dims=(arr_axis,))
        sign = torch.ones(3, dtype=torch.float64)
        sign[comp] = -1.0
        out = torch.cat([out, mirrored * sign], dim=arr_axis)
    return out


def energy_spectrum(u, nbins):
    """E(n) = sum_{round|k| = n} |u^(k)|^2 / 2 with u^ = FFT(u)/N^3 (oracle.diagnostics reading)."""
    nz, ny, nx = u.shape[:3]
    uh = torch.fft.fftn(u, dim=(0, 1, 2)) / (nx * ny * nz)
    e = 0.5 * (uh.real ** 2 + uh.imag ** 2).sum(-1)
    from .diagnostics import shell_index, wavenumbers
    kz, ky, kx = np.meshgrid(wavenumbers(nz), wavenumbers(ny), wavenumbers(nx), indexing="ij")
    shell = torch.tensor(shell_index(kx * kx + ky * ky + kz * kz).ravel())
    E = torch.zeros(nbins, dtype=torch.float64)
    keep = shell < nbins
    return E.index_add(0, shell[keep], e.reshape(-1)[keep])


def spectrum_loss(E, E_ref, kmin, kmax, omega, k_last):
    rel = (E[kmin: kmax + 1] - E_ref[kmin: kmax + 1]) / E_ref[kmin: kmax + 1]
    return (rel * rel).mean() + omega * E[k_last]
