"""FP64 CPU oracle of the solar-tomography hot path.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, obviously correct
restatement of what the projector, its transpose and the regularised
least-squares solver compute (TomograPy, Barbey, Guennou & Auchere; Eq. lo,
Eq. srt, Eq. criterion).  Only the test suite, the package smoke check and
the CPU-baseline leg of the benchmark may import it; the product path never
does.  It shares no code with the CUDA implementation; the two meet only
through the seeded inputs of the ``synth`` package.

Modules:
  siddon_oracle.c  FP64 merge-form Siddon, WCS ray reading, P, P^T (OpenMP)
  siddon.py        ctypes bindings of the C oracle
  checks.py        brute-force voxel clipping and fine sampling (pins)
  solver.py        finite-difference prior D, criterion J, textbook CG
  thomson.py       Thomson-scattering coefficients and the pB / B operators

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
against geometry, closed forms and brute force.  Agreement with the paper's
own software is unpinned: the paper prints no projector outputs.
"""

from . import siddon, checks, solver, thomson  # noqa: F401
