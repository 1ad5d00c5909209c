"""Write tgv64_re1600_nco_ke.txt: the FP64 oracle's kinetic-energy curve of the 64^3
Taylor-Green vortex at Re = 1600 stepped with the neural collision operator.

Setting (the underresolved case of the precision study): rho = 1, u = 0.05 (sin x cos y
cos z, -cos x sin y cos z, 0) on x_j = 2 pi j / 64, nu = 0.05 * 64 / (2 pi 1600),
equilibrium start, periodic box, network weights theta = Kaiming-uniform draws of seed 0
(lbm_inputs.nco_parameters). Fields and weights are first rounded to FP32, as the GPU
receives them. k = (1/2) <|u|^2> (Sec. IV.A reading) every 10 steps up to 400 steps
(about two convective times N / (2 pi U0)).

Calls only oracle/ and the seeded input generators. Run from the repository root:
    python tests/golden/make_tgv64_nco_ke.py
"""

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import lbm_inputs  # noqa: E402
from oracle import collision as col  # noqa: E402
from oracle import diagnostics as D  # noqa: E402
from oracle import stepper as S  # noqa: E402

N, U0, RE, STEPS, EVERY = 64, 0.05, 1600.0, 400, 10
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tgv64_re1600_nco_ke.txt")


def main():
    nu = lbm_inputs.reynolds_viscosity(U0, N, RE)
    rho, u = lbm_inputs.taylor_green_3d(N, U0)
    rho32 = rho.astype(np.float32).astype(np.float64)
    u32 = np.moveaxis(u.astype(np.float32).astype(np.float64), 0, -1)
    theta = lbm_inputs.nco_parameters(0).astype(np.float32).astype(np.float64)
    sim = S.Simulation.from_macroscopic(rho32, u32, col.tau_from_nu(nu), op="nco", theta=theta)
    rows = []
    t0 = time.time()
    for step in range(STEPS + 1):
        if step % EVERY == 0:
            _, uu = col.macroscopic(sim.f)
            rows.append((step, D.kinetic_energy(uu)))
            print(f"step {step} k {rows[-1][1]:.17e} ({time.time() - t0:.0f} s)", flush=True)
        if step < STEPS:
            sim.step(1)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle kinetic energy k = (1/2) <|u|^2> of the 64^3 Taylor-Green vortex, Re 1600,\n")
        fh.write(f"# NCO operator (seed-0 Kaiming weights, 27-20-20-4), nu = {nu:.17e}, U0 = {U0}, FP32-rounded start.\n")
        fh.write("# Written by tests/golden/make_tgv64_nco_ke.py (oracle/ only). Columns: step k\n")
        for step, k in rows:
            fh.write(f"{step} {k:.17e}\n")


if __name__ == "__main__":
    main()
