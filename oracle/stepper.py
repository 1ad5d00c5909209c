"""Streaming and the time loop of the lattice Boltzmann equation in FP64 (Sec. II.A).

Test infrastructure only (see the package docstring).

Populations are stored as arrays shaped (nz, ny, nx, 27). One step is
    f_i(x + c_i, t + 1) = f_i(x, t) + Omega_i(f) + S_i(f)        (Sec. II.A)
evaluated as: collide every cell, add the source, then stream.
"""

import numpy as np

from . import collision as col
from .lattice import C, Q


def stream_periodic(fstar):
    """Shift every population f*_i by c_i with periodic wrap (Sec. II.A, Sec. IV.C)."""
    out = np.empty_like(fstar)
    for i in range(Q):
        cx, cy, cz = C[i]
        out[..., i] = np.roll(fstar[..., i], shift=(cz, cy, cx), axis=(0, 1, 2))
    return out


def reflect_index(axis):
    """Velocity index map of the reflection S_axis (Appendix A): c -> c with component axis negated."""
    refl = np.empty(Q, dtype=np.int64)
    for i in range(Q):
        c = C[i].copy()
        c[axis] = -c[axis]
        refl[i] = int(np.where((C == c).all(axis=1))[0][0])
    return refl


def _pad_mirror(fstar):
    """Add one ghost layer on every face, each the mirror image of the adjacent layer.

    Nodes sit half a spacing from the symmetry planes, so the ghost at index -1
    is the reflection of layer 0 and the ghost at index N of layer N-1; the
    reflection also maps every population i to S_a(i) (Appendix A, matrices
    S_x, S_y, S_z). Padding axis by axis composes the reflections on edges and
    corners.
    """
    p = fstar
    # array axes are (z, y, x); velocity component index is (x, y, z)
    for arr_axis, comp in ((2, 0), (1, 1), (0, 2)):
        refl = reflect_index(comp)
        lo = np.take(p, [0], axis=arr_axis)[..., refl]
        hi = np.take(p, [p.shape[arr_axis] - 1], axis=arr_axis)[..., refl]
        p = np.concatenate([lo, p, hi], axis=arr_axis)
    return p


def stream_mirror(fstar):
    """Streaming on a mirror-symmetric box: specular reflection at all six faces.

    Reading for the octant [0, pi]^3 of the Taylor-Green vortex (Appendix A
    reduces the domain by its symmetries; on this octant only the reflections
    S_x, S_y, S_z apply): a population that would enter across a face comes from
    the mirrored population of the node next to the face.
    """
    p = _pad_mirror(fstar)
    nz, ny, nx = fstar.shape[:3]
    out = np.empty_like(fstar)
    for i in range(Q):
        cx, cy, cz = C[i]
        out[..., i] = p[1 - cz: 1 - cz + nz, 1 - cy: 1 - cy + ny, 1 - cx: 1 - cx + nx, i]
    return out


class Simulation:
    """The explicit time stepper: collide (+ Kupershtokh source), then stream.

    op: 'bgk', 'kbc', 'reg' or 'nco'; bc: 'periodic' or 'mirror'.
    ``forcing`` is an oracle.forcing.SpectralForcing or None.
    ``rates_override`` (4 values) replaces the network output of the NCO.
    """

    def __init__(self, f0, tau, op="bgk", theta=None, bc="periodic", forcing=None,
                 sizes=col.LAYER_SIZES, rates_override=None):
        self.f = np.array(f0, dtype=np.float64)
        self.tau = float(tau)
        self.op = op
        self.theta = None if theta is None else np.asarray(theta, dtype=np.float64)
        self.sizes = sizes
        self.bc = bc
        self.forcing = forcing
        self.rates_override = rates_override
        self.t = 0
        if forcing is not None:
            _, u = col.macroscopic(self.f)
            forcing.observe(u)

    @classmethod
    def from_macroscopic(cls, rho, u, tau, **kw):
        """Start from equilibrium populations f^eq(rho, u). rho: (nz,ny,nx), u: (nz,ny,nx,3)."""
        return cls(col.equilibrium(np.asarray(rho, float), np.asarray(u, float)), tau, **kw)

    def collide(self, f):
        if self.op == "bgk":
            return col.bgk(f, self.tau)
        if self.op == "kbc":
            return col.kbc_collide(f, self.tau)
        if self.op == "reg":
            return col.reg_collide(f, self.tau)
        if self.op == "nco":
            if self.rates_override is not None:
                rates = np.broadcast_to(np.asarray(self.rates_override, float), f.shape[:-1] + (4,))
            else:
                rates = col.nco_rates(f, self.theta, self.sizes)
            return col.mrt_collide(f, self.tau, rates)
        raise ValueError(self.op)

    def post_collision(self):
        """f* = f + Omega + S at the current time (before streaming)."""
        f = self.f
        fstar = self.collide(f)
        if self.forcing is not None:
            force = self.forcing.force_field(self.t, f.shape[:3])
            fstar = fstar + col.kupershtokh_source(f, force)
            _, u = col.macroscopic(f)
            self.forcing.observe(u)
        return fstar

    def step(self, n=1):
        for _ in range(n):
            fstar = self.post_collision()
            self.f = stream_periodic(fstar) if self.bc == "periodic" else stream_mirror(fstar)
            self.t += 1
        return self

    def macroscopic(self):
        return col.macroscopic(self.f)
