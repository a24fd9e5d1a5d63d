"""Parity over each workload's full horizon (Section 6 workloads' synthetic stand-ins).

* Neo-Hookean beam, 80x8x8 Q1 (19,683 DOFs), dt in {0.01, 0.02, 0.05, 0.1} against the oracle's
  stored trajectory (tests/golden/horizon_*.npz, written by tests/golden/make_horizon_goldens.py
  from the oracle alone): 500 / 200 / 50 / 30 steps. The horizons stop where the trajectory
  itself becomes unstable: with a 10% tip deflection the frozen-coefficient secant operator
  H(u*) is not symmetric and has complex eigenvalue pairs, so exp(dt A) amplifies some modes and
  the energy grows (to ~1e-2 at these step counts, in the oracle as on the GPU).
  FP64 with the oracle's Krylov sizes replayed: 1e-10 relative L2 in u and v; FP64 adaptive:
  1e-8; MIXED adaptive: u 1e-5; total energy every 10 steps (relative to the initial energy):
  FP64 1e-10, MIXED 1e-5 on the beam (its growing modes amplify the FP32 rounding: 4e-7 - 5e-6
  measured, against an energy growth of 8e-4 - 2e-2 in the trajectory itself).
  MIXED velocity: 1e-3 on the beam, 2e-4 elsewhere. The FP32 operator applied to a smooth
  displacement loses about eps_32 (omega_max / omega)^2 of H_bar u to cancellation in the
  element gradients and the node sums, so each step puts a velocity error of order
  eps_32 ||tau A|| (omega_max / omega) into the high modes; over these horizons that is
  1e-5 - 1e-4 of ||v|| (up to 7e-4 on the beam, whose growing modes amplify it), against
  1e-7 - 1e-6 for u and the energy. It is the MIXED form's arithmetic, not a defect: the FP64
  path holds 1e-10 on the same runs.
* Mooney-Rivlin slab 32x16x16 (28,611 DOFs, heterogeneous stiffness), 50 steps: same bars, MIXED
  energy 2e-6 (0.4 - 1.1e-6 measured; the coarse slab strains more than the full-size one, which
  meets the 1e-6 energy bar with 100x margin below).
* Q2 rubber cube 32^3 (823,875 DOFs), 200 steps: MIXED against the GPU FP64 path (itself
  pinned to the oracle above and on smaller Q2 meshes), u within 2e-5, energy within 1e-6, v
  within 2e-4 (as above).
* Mooney-Rivlin slab 256x128x128 (12,830,211 DOFs), 50 steps: MIXED against the GPU FP64 path,
  energy within 1e-6 relative, u within 1e-5, v within 2e-4.
With ETP_PARITY_REPORT set to a file name, every measured error is appended there as JSON.
"""
import json
import os

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def report(**rec):
    path = os.environ.get("ETP_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


@pytest.fixture(scope="module")
def E():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp
    assert torch.cuda.is_available()
    return etp, etp.Context(0)


def _golden(case):
    return np.load(os.path.join(HERE, "golden", f"horizon_{case}.npz"))


def _problem(case):
    if case.startswith("beam-neohooke-dt"):
        return inputs.beam_neohooke(dt=float(case[len("beam-neohooke-dt"):]), steps=500)
    return inputs.tissue_slab(nel=(32, 16, 16), steps=50)


def _run(etp, ctx, p, prec, steps, every, m_replay=None):
    mesh = etp.Mesh.from_problem(ctx, p)
    t = etp.Trajectory(mesh, p.u0, p.v0, prec, p.m_cap)
    energies = [t.energy()[0]]
    ms = []
    for k in range(steps):
        if m_replay is not None:
            st, info = t.step_ex(p.dt, p.tol, int(m_replay[2 * k]), int(m_replay[2 * k + 1]))
        else:
            st, info = t.step_ex(p.dt, p.tol)
        ms += [info.m_pred, info.m_corr]
        if (k + 1) % every == 0:
            energies.append(t.energy()[0])
    u, v = t.state()
    t.close()
    mesh.close()
    return u, v, np.array(energies), ms


CASES = ["beam-neohooke-dt0.01", "beam-neohooke-dt0.02", "beam-neohooke-dt0.05", "beam-neohooke-dt0.1",
         "tissue-mr-32x16x16"]


@pytest.mark.parametrize("case", CASES)
def test_horizon_against_oracle(E, case):
    etp, ctx = E
    g = _golden(case)
    p = _problem(case)
    steps, every = int(g["steps"]), int(g["energy_every"])
    assert float(g["dt"]) == p.dt and float(g["tol"]) == p.tol
    E0 = float(g["energy"][0])
    results = {}
    for name, prec, replay in (("fp64_replayed", etp.ETP_PREC_FP64, g["m"]),
                               ("fp64_adaptive", etp.ETP_PREC_FP64, None),
                               ("mixed_adaptive", etp.ETP_PREC_MIXED, None)):
        u, v, en, ms = _run(etp, ctx, p, prec, steps, every, replay)
        eu, ev = rel(u, g["u"]), rel(v, g["v"])
        de = float(np.max(np.abs(en - g["energy"])) / E0)
        same_m = float(np.mean(np.array(ms) == g["m"]))
        results[name] = (eu, ev, de)
        report(case=case, form=name, steps=steps, dt=p.dt, err_u=eu, err_v=ev, err_energy=de,
               energy_drift_oracle=float(abs(g["energy"][-1] - E0) / E0), m_agreement=same_m)
    eu, ev, de = results["fp64_replayed"]
    assert eu < 1e-10 and ev < 1e-10 and de < 1e-10, results
    eu, ev, de = results["fp64_adaptive"]
    assert eu < 1e-8 and ev < 1e-8 and de < 1e-8, results
    eu, ev, de = results["mixed_adaptive"]
    beam = case.startswith("beam")
    assert eu < 1e-5 and de < (1e-5 if beam else 2e-6) and ev < (1e-3 if beam else 2e-4), results


def _full_pair(etp, ctx, p, steps, every):
    """Run the FP64 and MIXED forms of p side by side; returns both end states and energies."""
    mesh = etp.Mesh.from_problem(ctx, p)
    out = {}
    for name, prec in (("fp64", etp.ETP_PREC_FP64), ("mixed", etp.ETP_PREC_MIXED)):
        t = etp.Trajectory(mesh, p.u0, p.v0, prec, p.m_cap)
        en = [t.energy()[0]]
        for k in range(steps):
            t.step(p.dt, p.tol)
            if (k + 1) % every == 0:
                en.append(t.energy()[0])
        out[name] = (*t.state(), np.array(en))
        t.close()
    mesh.close()
    return out


def test_rubber_q2_full_size_200_steps_mixed_vs_fp64(E):
    etp, ctx = E
    p = inputs.rubber_block()
    out = _full_pair(etp, ctx, p, p.steps, 20)
    u64, v64, e64 = out["fp64"]
    u32, v32, e32 = out["mixed"]
    eu, ev = rel(u32, u64), rel(v32, v64)
    de = float(np.max(np.abs(e32 - e64)) / e64[0])
    drift = float(abs(e64[-1] - e64[0]) / e64[0])
    report(case="rubber-neohooke-q2-823875dof", form="mixed_vs_fp64", steps=p.steps, dt=p.dt, err_u=eu,
           err_v=ev, err_energy=de, energy_drift_fp64=drift)
    assert eu < 2e-5 and de < 1e-6 and ev < 2e-4, (eu, ev, de)


def test_tissue_full_size_50_steps_mixed_vs_fp64(E):
    etp, ctx = E
    p = inputs.tissue_slab()
    out = _full_pair(etp, ctx, p, p.steps, 5)
    u64, v64, e64 = out["fp64"]
    u32, v32, e32 = out["mixed"]
    eu, ev = rel(u32, u64), rel(v32, v64)
    de = float(np.max(np.abs(e32 - e64)) / e64[0])
    drift = float(abs(e64[-1] - e64[0]) / e64[0])
    report(case="tissue-mooney-rivlin-q1-12830211dof", form="mixed_vs_fp64", steps=p.steps, dt=p.dt,
           err_u=eu, err_v=ev, err_energy=de, energy_drift_fp64=drift,
           energy_drift_mixed=float(abs(e32[-1] - e32[0]) / e32[0]))
    assert de < 1e-6, de
    assert eu < 1e-5 and ev < 2e-4, (eu, ev)
