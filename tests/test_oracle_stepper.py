"""Pins of oracle.stepper: streaming, viscous decay laws, step equivariance, octant BC (CPU only)."""

import math

import numpy as np
import pytest

import lbm_inputs
from oracle import collision as col
from oracle import lattice as L
from oracle import stepper as S
from oracle import diagnostics as D


def _aos(rho, u):
    """(nz,ny,nx) and (3,nz,ny,nx) -> (nz,ny,nx) and (nz,ny,nx,3)."""
    return rho, np.moveaxis(u, 0, -1)


def test_periodic_streaming_moves_each_population_by_its_velocity():
    n = 5
    for i in range(27):
        f = np.zeros((n, n, n, 27))
        f[1, 2, 3, i] = 1.0
        g = S.stream_periodic(f)
        cx, cy, cz = L.C[i]
        assert g[(1 + cz) % n, (2 + cy) % n, (3 + cx) % n, i] == 1.0
        assert g.sum() == 1.0


def test_mirror_streaming_reflects_at_faces():
    n = 4
    f = np.zeros((n, n, n, 27))
    i = int(np.where((L.C == [-1, 0, 0]).all(axis=1))[0][0])  # moving in -x
    f[2, 1, 0, i] = 1.0
    g = S.stream_mirror(f)
    j = L.OPP[i]
    assert g[2, 1, 0, j] == 1.0 and g.sum() == 1.0  # comes back in +x at the same node
    # corner: (-1,-1,-1) at the corner node returns as (+1,+1,+1)
    f = np.zeros((n, n, n, 27))
    f[0, 0, 0, 0] = 1.0
    g = S.stream_mirror(f)
    assert g[0, 0, 0, 26] == 1.0 and g.sum() == 1.0


def _fit_rate(values):
    t = np.arange(len(values))
    return -np.polyfit(t, np.log(values), 1)[0]


@pytest.mark.parametrize("op", ["bgk", "nco"])
def test_shear_wave_decays_at_lattice_viscosity(op):
    """u_x = U0 sin(k y) decays as exp(-nu k^2 t) with nu = cs^2 (tau - 1/2) (Sec. II.B)."""
    n, nu, u0 = 32, 0.04, 1e-3
    tau = col.tau_from_nu(nu)
    rho, u = _aos(*lbm_inputs.shear_wave(n, u0))
    sim = S.Simulation.from_macroscopic(rho, u, tau, op=op, theta=lbm_inputs.nco_parameters(0))
    k = 2 * math.pi / n
    amps = []
    for _ in range(120):
        _, uu = sim.macroscopic()
        amps.append(np.abs(np.fft.fft(uu[0, :, 0, 0]))[1])
        sim.step()
    nu_meas = _fit_rate(np.array(amps[20:])) / (k * k)
    assert nu_meas == pytest.approx(nu, rel=1e-2)


def test_taylor_green_2d_decay():
    """2-D Taylor-Green: u ~ exp(-2 nu kappa^2 t), kappa = 2 pi / N (Sec. III.B)."""
    n, nu, u0 = 32, 0.02, 1e-3
    rho, u = _aos(*lbm_inputs.taylor_green_2d(n, u0))
    sim = S.Simulation.from_macroscopic(rho, u, col.tau_from_nu(nu))
    kap = 2 * math.pi / n
    ke = []
    for _ in range(100):
        ke.append(D.kinetic_energy(sim.macroscopic()[1]))
        sim.step()
    rate = _fit_rate(np.sqrt(np.array(ke[10:])))
    assert rate == pytest.approx(2 * nu * kap * kap, rel=1e-2)


def test_taylor_green_3d_low_re_energy_decay_converges_second_order():
    """Low-Re 3-D Taylor-Green: k ~ exp(-6 nu kappa^2 t); the lattice error halves twice per refinement.

    Sec. III.B expects the operator to converge with resolution; at Re ~ 0.3 the
    nonlinear transfer is negligible and the decay rate is the viscous one.
    """
    errs = []
    for n in (16, 32):
        nu, u0 = 0.05, 0.005
        rho, u = _aos(*lbm_inputs.taylor_green_3d(n, u0))
        sim = S.Simulation.from_macroscopic(rho, u, col.tau_from_nu(nu))
        kap = 2 * math.pi / n
        ke = []
        for _ in range(60):
            ke.append(D.kinetic_energy(sim.macroscopic()[1]))
            sim.step()
        rate = _fit_rate(np.array(ke[10:]))
        errs.append(abs(rate / (6 * nu * kap * kap) - 1.0))
    assert errs[0] < 2.5e-2 and errs[1] < 1e-2
    assert 3.0 < errs[0] / errs[1] < 5.0


def _transform_field(f, g):
    """(T_g f)_{pi(i)}(R x) = f_i(x) on a periodic N^3 grid (indices taken mod N)."""
    n = f.shape[0]
    R = L.G_MATRICES[g]
    p = L.G_VPERM[g]
    out = np.empty_like(f)
    idx = np.indices((n, n, n)).reshape(3, -1)  # (z, y, x)
    xyz = idx[::-1]  # (x, y, z)
    new = (R @ xyz) % n
    out_pop = np.empty_like(f)
    out_pop[..., p] = f  # population i goes to pi(i)
    out[new[2], new[1], new[0]] = out_pop[idx[0], idx[1], idx[2]]
    return out


@pytest.mark.parametrize("op", ["nco", "kbc"])
def test_full_step_equivariance_under_all_48_elements(op):
    """Step(T_g f) = T_g Step(f) for all g in O_h on a 4^3 periodic grid (Sec. II.B)."""
    f0 = np.moveaxis(lbm_inputs.random_populations((4, 4, 4), 21), 0, -1)
    theta = lbm_inputs.nco_parameters(0)
    def step(f):
        return S.Simulation(f, 0.56, op=op, theta=theta).step(1).f
    base = step(f0)
    for g in range(48):
        lhs = step(_transform_field(f0, g))
        rhs = _transform_field(base, g)
        assert np.allclose(lhs, rhs, atol=1e-15), g


def test_nco_with_pinned_rates_matches_bgk_over_many_steps():
    rho, u = _aos(*lbm_inputs.taylor_green_3d(8, 0.05))
    tau = 0.6
    a = S.Simulation.from_macroscopic(rho, u, tau, op="nco", rates_override=[1 / tau] * 4).step(10)
    b = S.Simulation.from_macroscopic(rho, u, tau, op="bgk").step(10)
    assert np.allclose(a.f, b.f, atol=1e-15)


def test_octant_with_mirror_boundaries_equals_full_periodic_domain():
    """A BGK run on the mirror octant equals the octant of the full periodic run (Appendix A)."""
    n = 6
    tau = 0.56
    rho_o, u_o = _aos(*lbm_inputs.taylor_green_octant(n, 0.05))
    rho_f, u_f = _aos(*lbm_inputs.taylor_green_3d(2 * n, 0.05, shifted=True))
    oct_sim = S.Simulation.from_macroscopic(rho_o, u_o, tau, bc="mirror").step(12)
    full = S.Simulation.from_macroscopic(rho_f, u_f, tau).step(12)
    assert np.allclose(oct_sim.f, full.f[:n, :n, :n], atol=1e-15)
    # and for the neural operator, whose equivariance makes it commute with the mirrors
    theta = lbm_inputs.nco_parameters(0)
    oct_sim = S.Simulation.from_macroscopic(rho_o, u_o, tau, bc="mirror", op="nco", theta=theta).step(3)
    full = S.Simulation.from_macroscopic(rho_f, u_f, tau, op="nco", theta=theta).step(3)
    assert np.allclose(oct_sim.f, full.f[:n, :n, :n], atol=1e-15)
