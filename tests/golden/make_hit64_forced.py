"""Write hit64_forced_<op>.txt: the FP64 oracle's kinetic-energy curve and energy spectra
of forced isotropic turbulence on a 64^3 periodic box over its first 1000 steps, for the
BGK and the neural collision operator.

Setting (the forced-turbulence workload, Sec. II.C forcing): the seeded isotropic field of
lbm_inputs.isotropic_field(64, seed 1, u_rms 0.04) (E(k) ~ k^4 exp(-2 (k/4)^2), rho = 1),
nu = 0.0015, the spectral force on the 16 half-space modes 1 <= |k| <= 2 with the random
phases lbm_inputs.forcing_draws(1000, seed 1) and the power input P = nu <|grad u|^2> of the
initial field (numpy central differences). Fields are rounded to FP32 first, as the GPU
receives them; the start is the equilibrium of (rho, u). NCO weights: Kaiming-uniform draws
of seed 0 (lbm_inputs.nco_parameters).

Recorded: k = (1/2) <|u|^2> every 10 steps and the energy spectrum E(n)
(oracle.diagnostics.energy_spectrum, Sec. II.D) every 100 steps.

Each step is oracle.stepper.Simulation.step: collision, the Kupershtokh source of the force
synthesised from the previous velocity's projection, periodic streaming. For the neural
operator the per-cell rates (oracle.collision.nco_rates) are evaluated on z-slabs in a pool
of worker processes; this changes which rows one library call sees, nothing else. Calls
only oracle/ and the seeded input generators. Run from the repository root:
    python tests/golden/make_hit64_forced.py bgk|nco [--workers W]
(BGK a few minutes; NCO about half an hour on 8 cores).
"""

import argparse
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

N, NU, URMS, SEED, STEPS, EVERY, SPECTRUM_EVERY = 64, 0.0015, 0.04, 1, 1000, 10, 100

_w = {}


def _worker_init(theta):
    sys.path.insert(0, ROOT)
    _w["theta"] = theta


def _rates_slab(f_slab):
    from oracle import collision as col
    return col.nco_rates(f_slab, _w["theta"])


def forcing_power(u):
    """P = nu <|grad u|^2> of the initial field (central differences, lattice units)."""
    import numpy as np
    grads = [np.gradient(u[a], axis=ax) for a in range(3) for ax in range(3)]
    return float(NU * np.mean(sum(g * g for g in grads)))


def main():
    sys.path.insert(0, ROOT)
    import numpy as np
    import lbm_inputs
    from oracle import collision as col
    from oracle import diagnostics as D
    from oracle import forcing as F
    from oracle import stepper as S

    ap = argparse.ArgumentParser()
    ap.add_argument("op", choices=["bgk", "nco"])
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    args = ap.parse_args()

    rho, u = lbm_inputs.isotropic_field(N, SEED, URMS)
    rho = rho.astype(np.float32).astype(np.float64)
    u = u.astype(np.float32).astype(np.float64)
    power = forcing_power(u)
    phi, psi = lbm_inputs.forcing_draws(STEPS, seed=SEED)
    theta = lbm_inputs.nco_parameters(0).astype(np.float32).astype(np.float64)
    tau = col.tau_from_nu(NU)
    forcing = F.SpectralForcing(phi, psi, power=power)
    sim = S.Simulation.from_macroscopic(rho, np.moveaxis(u, 0, -1), tau, op=args.op,
                                        theta=theta if args.op == "nco" else None, forcing=forcing)
    pool = None
    if args.op == "nco":
        # one BLAS thread per worker (the spawned workers read this when they import numpy)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        pool = mp.get_context("spawn").Pool(args.workers, initializer=_worker_init, initargs=(theta,))
        slabs = [(z, min(z + 2, N)) for z in range(0, N, 2)]

        def collide(f):
            rates = np.concatenate(pool.map(_rates_slab, [f[z0:z1] for z0, z1 in slabs]), axis=0)
            return col.mrt_collide(f, tau, rates)

        sim.collide = collide

    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"hit64_forced_{args.op}.txt")
    lines = [f"# FP64 oracle of forced isotropic turbulence 64^3 ({args.op}), seed {SEED}, u_rms {URMS},",
             f"# nu = {NU!r}, power = {power!r}, forcing draws of seed {SEED}, FP32-rounded start, {STEPS} steps.",
             "# Written by tests/golden/make_hit64_forced.py (oracle/ only).",
             "# Rows 'k step value': k = (1/2) <|u|^2>. Rows 'E step E(0) E(1) ...': energy spectrum."]

    def record(t):
        _, uu = sim.macroscopic()
        lines.append(f"k {t} {D.kinetic_energy(uu)!r}")
        if t % SPECTRUM_EVERY == 0:
            E = D.energy_spectrum(uu)
            lines.append(f"E {t} " + " ".join(repr(float(e)) for e in E))

    t0 = time.time()
    record(0)
    for t in range(1, STEPS + 1):
        sim.step(1)
        if t % EVERY == 0:
            record(t)
        if t % 100 == 0:
            print(f"step {t} ({time.time() - t0:.0f} s)", flush=True)
    if pool is not None:
        pool.close()
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
