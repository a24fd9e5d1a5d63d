"""FP64 CPU oracle of the exponential time propagator (arXiv 2405.05213).

TEST INFRASTRUCTURE, NOT PRODUCT. This package is the plain, slow, obviously
correct reference that the CUDA path is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import or run it; the library under ``paper_2405_05213_gb300/`` never does, and
the two share no code (only the seeded generators in ``inputs/``).

Modules:
  fem         hexahedral Q1/Q2 discretisation, GLL mass, assembled H(u*)
  materials   constitutive laws and the secant split P_lin
  expm        Pade [13/13] scaling and squaring; Taylor "direct exponentiation"
  krylov      Arnoldi (CGS2) evaluation of exp(tau A) w with the a-priori estimate
  propagator  the Magnus midpoint step with predictor-corrector, energy
  newmark     Newmark-beta (beta=1/4, gamma=1/2), the paper's comparison method

Parity status per function: every function here is pinned by a test in
``tests/test_oracle_*.py`` against closed forms, invariants or library
routines. Nothing is "parity unpinned" except the nonlinear propagator's
agreement with the paper's own runs (the paper's meshes and material data are
not given).
"""
