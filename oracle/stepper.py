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
    """Shift every population f*_i by c_i with periodic wrap (Sec. II.A, Sec. III.C)."""
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


# --- the reduced Taylor-Green domain [0, pi/2]^3 (Appendix A) ----------------------------


def _tgv_velocity(p):
    """Velocity field of the 3-D Taylor-Green vortex (Sec. III.C, Eq. tgv3d), unit amplitude."""
    x, y, z = p[..., 0], p[..., 1], p[..., 2]
    return np.stack([np.sin(x) * np.cos(y) * np.cos(z), -np.cos(x) * np.sin(y) * np.cos(z), 0.0 * x], -1)


def tgv_symmetry_group():
    """The symmetries (A, t) of the Taylor-Green field, u(A x + t) = A u(x), with A a signed
    permutation matrix (a symmetry of the D3Q27 lattice) and t in (pi/2) Z^3 modulo 2 pi.

    Found by checking every candidate on random points: the flow's rotations, reflections
    and the x-y exchanges the Appendix A tables use (S_a, R_b, T_xy). Returns a list of
    (A, k) with A a 3 x 3 integer matrix and k the translation in units of pi/2 (0..3).
    """
    import itertools
    rng = np.random.default_rng(0)
    pts = rng.uniform(0.0, 2 * np.pi, (256, 3))
    group = []
    for perm in itertools.permutations(range(3)):
        for sgn in itertools.product((1, -1), repeat=3):
            A = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                A[r, perm[r]] = sgn[r]
            for k in itertools.product(range(4), repeat=3):
                t = np.array(k) * (np.pi / 2)
                if np.allclose(_tgv_velocity(pts @ A.T + t), _tgv_velocity(pts) @ A.T, atol=1e-12):
                    group.append((A, np.array(k, dtype=np.int64)))
    return group


def _velocity_index(c):
    return int(np.where((C == c).all(axis=1))[0][0])


def stream_tgv_reduced(fstar, group=None):
    """Streaming on the reduced Taylor-Green domain [0, pi/2]^3 with N nodes per axis at
    (j + 1/2) pi / (2N) (Appendix A): a population whose source x - c_i lies outside the
    domain is taken from the node g(x - c_i) inside it, with the velocity index of A c_i,
    where g = (A, t) is the symmetry of the flow that maps the source's block (of the
    tiling of the periodic box by the 64 images of the domain) back onto the domain.
    Coordinates are doubled units of h = pi / (2N): node j sits at 2j + 1; t is a multiple
    of 2N, all modulo 8N.
    """
    group = tgv_symmetry_group() if group is None else group
    n = fstar.shape[0]
    assert fstar.shape[:3] == (n, n, n), "the reduced domain is a cube"
    out = np.empty_like(fstar)
    idx = np.arange(n)
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    for i in range(Q):
        c = C[i]
        src = np.stack([X - c[0], Y - c[1], Z - c[2]], -1)          # (x, y, z) indices
        inside = ((src >= 0) & (src < n)).all(-1)
        vals = np.empty(X.shape)
        s_in = src[inside]
        vals[inside] = fstar[s_in[:, 2], s_in[:, 1], s_in[:, 0], i]
        for pt in np.argwhere(~inside):
            sp = src[tuple(pt)]
            found = False
            for A, k in group:
                img = (A @ (2 * sp + 1) + 2 * n * k) % (8 * n)
                j = (img - 1) // 2
                if ((j >= 0) & (j < n)).all():
                    vals[tuple(pt)] = fstar[j[2], j[1], j[0], _velocity_index(A @ c)]
                    found = True
                    break
            assert found
        out[..., i] = vals
    return out


class Simulation:
    """The explicit time stepper: collide (+ Kupershtokh source), then stream.

    op: 'bgk', 'kbc', 'reg' or 'nco'; bc: 'periodic', 'mirror' or 'tgv_reduced'.
    ``forcing`` is an oracle.forcing.SpectralForcing or None.
    ``rates_override`` (4 values) replaces the network output of the NCO.
    ``operand_round`` is passed to the network (oracle.collision.phi_network; default exact).
    """

    def __init__(self, f0, tau, op="bgk", theta=None, bc="periodic", forcing=None,
                 sizes=col.LAYER_SIZES, rates_override=None, operand_round=None):
        self.f = np.array(f0, dtype=np.float64)
        self.tau = float(tau)
        self.op = op
        self.theta = None if theta is None else np.asarray(theta, dtype=np.float64)
        self.sizes = sizes
        self.bc = bc
        self.forcing = forcing
        self.rates_override = rates_override
        self.operand_round = operand_round
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
                rates = col.nco_rates(f, self.theta, self.sizes, operand_round=self.operand_round)
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
            if self.bc == "periodic":
                self.f = stream_periodic(fstar)
            elif self.bc == "mirror":
                self.f = stream_mirror(fstar)
            elif self.bc == "tgv_reduced":
                self.f = stream_tgv_reduced(fstar, self._group())
            else:
                raise ValueError(self.bc)
            self.t += 1
        return self

    def macroscopic(self):
        return col.macroscopic(self.f)

    def _group(self):
        if not hasattr(self, "_tgv_group"):
            self._tgv_group = tgv_symmetry_group()
        return self._tgv_group
