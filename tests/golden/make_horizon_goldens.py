"""Write the oracle's full-horizon trajectories used by the GPU horizon parity tests.

Only ``oracle/`` and the seeded generators in ``inputs/`` are called: every stored
value is the FP64 oracle's. Each case stores the final physical state (u, v), the
Krylov size of every solve (predictor and corrector, in order), the step's error
estimate and the total energy every ``energy_every`` steps.

Cases (Section 6 workloads' synthetic stand-ins):
  beam-neohooke-dt{0.01,0.02,0.05,0.1}  Neo-Hookean Q1 beam 80x8x8 (19,683 DOFs),
                                        500 / 200 / 50 / 30 steps (HORIZON), tol 1e-8
  tissue-mr-32x16x16                    Mooney-Rivlin Q1 slab 32x16x16 (28,611 DOFs)
                                        with the heterogeneous element scale, 50 steps,
                                        tol 1e-6, dt of the full-size slab's rule

Usage: python tests/golden/make_horizon_goldens.py CASE [CASE ...]   (about 15-20 min
per beam case, 3 min for the slab, on one core each; the cases are independent).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import inputs  # noqa: E402
from oracle import propagator  # noqa: E402


def problem(case):
    if case.startswith("beam-neohooke-dt"):
        dt = float(case[len("beam-neohooke-dt"):])
        return inputs.beam_neohooke(dt=dt, steps=HORIZON[dt]), 10
    if case == "tissue-mr-32x16x16":
        return inputs.tissue_slab(nel=(32, 16, 16), steps=50), 1
    raise ValueError(case)


# Steps stored per dt of the beam: 500, or fewer where the trajectory is unstable. With a 10%
# tip deflection the frozen-coefficient secant operator H(u*) is not symmetric (its relative
# skew part grows to ~1e-2) and has complex eigenvalue pairs, so exp(dt A) amplifies some modes
# and the energy grows; the stored horizon ends before the energy error reaches ~1e-2 (the
# oracle's own trajectory; at dt 0.02, 0.05 and 0.1 an element inverts later on).
HORIZON = {0.01: 500, 0.02: 200, 0.05: 50, 0.1: 30}

CASES = ["beam-neohooke-dt0.01", "beam-neohooke-dt0.02", "beam-neohooke-dt0.05",
         "beam-neohooke-dt0.1", "tissue-mr-32x16x16"]


def path_of(case):
    return os.path.join(HERE, f"horizon_{case}.npz")


def make(case):
    p, every = problem(case)
    P = propagator.Propagator.from_problem(p)
    energies = [P.energy()[0]]
    t0 = time.time()
    for k in range(p.steps):
        P.step(p.dt, p.tol)
        if (k + 1) % every == 0:
            energies.append(P.energy()[0])
    np.savez_compressed(path_of(case), u=P.u_full(), v=P.v_full(),
                        m=np.asarray(P.log.m, dtype=np.int32),
                        eps=np.asarray(P.log.eps, dtype=np.float64),
                        converged=np.asarray(P.log.converged, dtype=bool),
                        energy=np.asarray(energies), energy_every=every,
                        dt=p.dt, tol=p.tol, steps=p.steps)
    print(f"{case}: {p.steps} steps in {time.time() - t0:.0f} s, m max {max(P.log.m)}, "
          f"energy drift {abs(energies[-1] - energies[0]) / energies[0]:.2e}", flush=True)


if __name__ == "__main__":
    for c in (sys.argv[1:] or CASES):
        make(c)
