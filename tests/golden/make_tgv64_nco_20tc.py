"""Write tgv64_re1600_nco_20tc.txt: the FP64 oracle's kinetic-energy curve and energy
spectra of the 64^3 Taylor-Green vortex at Re = 1600 over 20 convective times, stepped with
the neural collision operator.

Setting (the underresolved case of the precision study, Sec. III.C flow): rho = 1,
u = 0.05 (sin x cos y cos z, -cos x sin y cos z, 0) on x_j = 2 pi j / 64,
nu = 0.05 * 64 / (2 pi 1600), equilibrium start, periodic box, network weights theta =
Kaiming-uniform draws of seed 0 (lbm_inputs.nco_parameters). Fields and weights are first
rounded to FP32, as the GPU receives them. One convective time is N / (2 pi U0) = 203.7
steps, so 4080 steps cover 20.03 of them.

Recorded: k = (1/2) <|u|^2> (Sec. IV.A reading) every 10 steps, and the energy spectrum
E(n) (oracle.diagnostics.energy_spectrum, Sec. II.D) every 1020 steps.

Each step is oracle.collision.nco_collide on every cell followed by
oracle.stepper.stream_periodic, exactly as oracle.stepper.Simulation steps it. The
collision is a per-cell map, so it is evaluated on z-slabs in a pool of worker processes
that write into shared memory; this changes which rows one library call sees, nothing else.
Calls only oracle/ and the seeded input generators. Run from the repository root:
    python tests/golden/make_tgv64_nco_20tc.py [--workers W] [--checkpoint PATH]
(about 1.5 to 2 hours on 6 cores). --checkpoint saves the state every 200 steps and resumes
from it.
"""

import argparse
import multiprocessing as mp
import os
import sys
import time
from multiprocessing import shared_memory

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

N, U0, RE, STEPS, EVERY, SPECTRUM_EVERY = 64, 0.05, 1600.0, 4080, 10, 1020
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tgv64_re1600_nco_20tc.txt")
SHAPE = (N, N, N, 27)

_w = {}


def _worker_init(name_f, name_out, tau, theta):
    sys.path.insert(0, ROOT)
    import numpy as np
    _w["shm"] = (shared_memory.SharedMemory(name=name_f), shared_memory.SharedMemory(name=name_out))
    _w["f"] = np.ndarray(SHAPE, dtype=np.float64, buffer=_w["shm"][0].buf)
    _w["out"] = np.ndarray(SHAPE, dtype=np.float64, buffer=_w["shm"][1].buf)
    _w["tau"], _w["theta"] = tau, theta


def _collide_slab(z0z1):
    from oracle import collision as col
    z0, z1 = z0z1
    _w["out"][z0:z1] = col.nco_collide(_w["f"][z0:z1], _w["tau"], _w["theta"])
    return z0


def main():
    sys.path.insert(0, ROOT)
    import numpy as np
    import lbm_inputs
    from oracle import collision as col
    from oracle import diagnostics as D
    from oracle import stepper as S

    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--checkpoint", default=None)
    args = ap.parse_args()

    nu = lbm_inputs.reynolds_viscosity(U0, N, RE)
    tau = col.tau_from_nu(nu)
    theta = lbm_inputs.nco_parameters(0).astype(np.float32).astype(np.float64)
    shm_f = shared_memory.SharedMemory(create=True, size=int(np.prod(SHAPE)) * 8)
    shm_o = shared_memory.SharedMemory(create=True, size=int(np.prod(SHAPE)) * 8)
    f = np.ndarray(SHAPE, dtype=np.float64, buffer=shm_f.buf)
    fstar = np.ndarray(SHAPE, dtype=np.float64, buffer=shm_o.buf)

    ke_rows, spec_rows, start = [], [], 0
    if args.checkpoint and os.path.exists(args.checkpoint):
        ck = np.load(args.checkpoint, allow_pickle=False)
        f[...] = ck["f"]
        start = int(ck["step"])
        ke_rows = [tuple(r) for r in ck["ke"]]
        spec_rows = [(int(r[0]), r[1:]) for r in ck["spec"]]
        print(f"resumed at step {start}", flush=True)
    else:
        rho, u = lbm_inputs.taylor_green_3d(N, U0)
        rho32 = rho.astype(np.float32).astype(np.float64)
        u32 = np.moveaxis(u.astype(np.float32).astype(np.float64), 0, -1)
        f[...] = col.equilibrium(rho32, u32)

    slabs = [(z, min(z + 2, N)) for z in range(0, N, 2)]
    # one BLAS thread per worker: the workers inherit this environment and read it when
    # they first import numpy (unpickling their arguments), before any initializer runs
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(args.workers, initializer=_worker_init,
                  initargs=(shm_f.name, shm_o.name, tau, theta)) as pool:
        for step in range(start, STEPS + 1):
            if step % EVERY == 0 and (not ke_rows or ke_rows[-1][0] < step):
                _, uu = col.macroscopic(f)
                ke_rows.append((step, D.kinetic_energy(uu)))
                if step % SPECTRUM_EVERY == 0:
                    spec_rows.append((step, D.energy_spectrum(uu)))
                print(f"step {step} k {ke_rows[-1][1]:.17e} ({time.time() - t0:.0f} s)", flush=True)
            if step == STEPS:
                break
            for _ in pool.imap_unordered(_collide_slab, slabs):
                pass
            f[...] = S.stream_periodic(fstar)
            if args.checkpoint and (step + 1) % 200 == 0:
                tmp = args.checkpoint + ".tmp.npz"
                np.savez(tmp, f=f, step=step + 1, ke=np.array(ke_rows),
                         spec=np.array([np.concatenate([[s], e]) for s, e in spec_rows]))
                os.replace(tmp, args.checkpoint)

    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle of the 64^3 Taylor-Green vortex, Re 1600, NCO operator (seed-0 Kaiming\n")
        fh.write(f"# weights, 27-20-20-4), nu = {nu:.17e}, U0 = {U0}, FP32-rounded start, {STEPS} steps.\n")
        fh.write("# Written by tests/golden/make_tgv64_nco_20tc.py (oracle/ only).\n")
        fh.write("# Rows 'k step value': k = (1/2) <|u|^2>. Rows 'E step E(0) E(1) ...': energy spectrum.\n")
        for step, k in ke_rows:
            fh.write(f"k {int(step)} {k:.17e}\n")
        for step, e in spec_rows:
            fh.write(f"E {int(step)} " + " ".join(f"{v:.17e}" for v in e) + "\n")
    shm_f.close()
    shm_f.unlink()
    shm_o.close()
    shm_o.unlink()


if __name__ == "__main__":
    main()
