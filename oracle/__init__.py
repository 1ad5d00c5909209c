"""FP64 CPU oracle for the D3Q27 neural-collision lattice Boltzmann step.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
or run anything in this package. The CUDA library never calls it and shares no
code, table or constant generator with it.

Everything here is a plain, slow, step-by-step restatement of arXiv 2412.08229
(Bedrunka et al., "Machine Learning Enhanced Collision Operator for the Lattice
Boltzmann Method Based on Invariant Networks") in float64 NumPy. Each function
cites the section / equation it follows. Where the paper is silent or garbled
the reading taken is stated in the docstring.

Modules
  lattice      D3Q27 velocities and weights, Hermite moment matrix M, the
               octahedral group O_h acting on velocities and moments.
  collision    equilibrium, BGK, the neural collision operator (NCO), KBC,
               Kupershtokh forcing.
  stepper      periodic and mirror-octant streaming, the time loop.
  forcing      Alvelius spectral forcing.
  diagnostics  kinetic energy, dissipation, energy spectrum, spectrum loss.

Parity status per function (what pins it, see tests/test_oracle_*.py):
  all functions are pinned by closed forms, invariants or brute force, except
  the absolute behaviour of a *trained* NCO, which is parity unpinned because
  the paper's trained weights are not available (only the architecture is).
"""

from . import lattice, collision, stepper, forcing, diagnostics  # noqa: F401
