"""Throughput benchmark of the exponential time propagator on GB300.

One step = one time step of the propagator (Section 3-4 of arXiv 2405.05213):
for a nonlinear material the predictor solve, the midpoint operator and the
corrector solve, each an adaptive Arnoldi process with CGS2 and the small
exponential, through the C ABI of libetp.

Workload (default): the soft-tissue slab, 2x1x1 box meshed with 256x128x128 Q1
hexahedra (12,830,211 DOFs), Mooney-Rivlin C10=0.5, C01=0.05, kappa=1.1e3,
lognormal per-element stiffness exp(0.1 N(0,1)), x=0 fixed, seeded velocity
patch at x=2, dt = 6 h / c_p, 50-step horizon, Krylov tol 1e-6, m_cap 64; FP32
operator and basis with FP64 reductions, exponential and state. The largest
configuration: its vectors (102 MB each) and basis (GBs) stream from HBM, which
is where the metric's roofline is defined. Other workloads: --workload.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the library's stream, with an L2 flush (a 512 MiB write) between steps and
outside the events; barrier + synchronize on both sides; max over ranks.
Multi-GPU: one independent replica per rank (weak scaling, no collective on
the data path).

--impl reference times the FP64 CPU oracle (the only reference this project
has) on the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF·steps/s and % HBM roofline; served p50/p99 step latency vs plain FP64"
UNIT = "DOF·steps/s"

WORKLOADS = {
    # name: (problem factory kwargs, precision)
    "beam-neohooke-q1-19683dof": ("beam-neohooke-q1", {"dt": 0.02}, "mixed"),
    "beam-neohooke-q1-19683dof-fp64": ("beam-neohooke-q1", {"dt": 0.02}, "fp64"),
    "rubber-neohooke-q2-823875dof": ("rubber-neohooke-q2", {}, "mixed"),
    "tissue-mooney-rivlin-q1-12830211dof": ("tissue-mooney-rivlin-q1", {}, "mixed"),
    # a 128x64x64 slab (1,622,595 DOFs): the same kernels at a size ncu captures in full
    "tissue-mooney-rivlin-q1-1622595dof": ("tissue-mooney-rivlin-q1", {"nel": (128, 64, 64)}, "mixed"),
    "beam-linear-q1-567dof": ("beam-linear-q1", {}, "fp64"),
    # constant external load (the augmented state of Eq. "A expression at P != 0"):
    # a total force on the x = max face, split over its free nodes
    "beam-neohooke-q1-19683dof-loaded": ("beam-neohooke-q1", {"dt": 0.02, "face_load": (-2.0, 1)}, "mixed"),
    "tissue-mooney-rivlin-q1-12830211dof-loaded": ("tissue-mooney-rivlin-q1", {"face_load": (-0.01, 0)}, "mixed"),
    # the same slab with a linear material of the same small-strain moduli: the workload of the
    # energy Lanczos process (--krylov lanczos) against Arnoldi
    "tissue-linear-q1-12830211dof": ("tissue-mooney-rivlin-q1", {"linear": True}, "mixed"),
}


def make_workload_problem(name):
    """The synthetic problem of a bench workload (with its load, if any)."""
    import inputs
    pname, pkw, precision = WORKLOADS[name]
    pkw = dict(pkw)
    fl = pkw.pop("face_load", None)
    linear = pkw.pop("linear", False)
    prob = inputs.make_problem(pname, **pkw)
    if linear:
        lam, mu = inputs.small_strain_moduli(prob.material, prob.params)
        prob.material = inputs.MAT_LINEAR
        prob.params = (mu * (3 * lam + 2 * mu) / (lam + mu), lam / (2 * (lam + mu)))
        prob.name = prob.name.replace("mooney-rivlin", "linear")
    if fl is not None:
        prob = inputs.with_face_load(prob, fl[0], comp=fl[1])
    return prob, precision
# The largest configuration: the one whose kernels stream from HBM (the metric's
# roofline is defined there); the beam and block workloads remain selectable.
DEFAULT_WORKLOAD = "tissue-mooney-rivlin-q1-12830211dof"
# Oracle samples for workloads too large for whole oracle steps in ~15 s: the same
# problem on a coarser mesh with the same dt/h ratio (hence the same Krylov sizes).
# Candidates from largest to smallest; the largest whose oracle step fits the time
# budget is used (the oracle runs ~7.5e3 DOF-steps/s on these).
ORACLE_SAMPLE = {
    "tissue-mooney-rivlin-q1-12830211dof": ("tissue-mooney-rivlin-q1", [{"nel": (32, 16, 16)},
                                                                        {"nel": (24, 12, 12)},
                                                                        {"nel": (16, 8, 8)}]),
    "tissue-mooney-rivlin-q1-1622595dof": ("tissue-mooney-rivlin-q1", [{"nel": (32, 16, 16)},
                                                                       {"nel": (16, 8, 8)}]),
    "rubber-neohooke-q2-823875dof": ("rubber-neohooke-q2", [{"n": 8}, {"n": 4}]),
}
ORACLE_DOF_STEPS_PER_S = 7.5e3


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _fp32_peak_tflops():
    """Dense FP32 FMA peak from unit counts and clocks: SMs x 128 lanes x 2 x max SM clock."""
    try:
        import torch
        sms = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        sms = 152
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", 2070.0))
    except Exception:
        mhz = 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12


# Sources that define each kernel class whose DRAM counters profiles/dram_traffic.json holds (the
# counters stand while these files are unchanged); any other class: every library source.
KERNEL_SOURCES = {"elem_apply": ["etp_internal.cuh", "fe_dispatch.cuh", "fe_kernels.cuh", "fe_q1_f32.cu",
                                 "material.cuh"]}


def _src_hash(kernel=None):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2405_05213_gb300", "csrc")
    names = KERNEL_SOURCES.get(kernel) or sorted(os.listdir(d))
    for n in sorted(names):
        with open(os.path.join(d, n), "rb") as f:
            h.update(n.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it matches this source."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            t = json.load(f)
        e = t[workload][kernel]
        if e.get("src_hash") != _src_hash(kernel):
            return None
        return float(e["bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the warm-up and the timed region
    (every 200 ms)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_problem(prob, wl_name, seconds_per_step=5.0):
    """(problem the oracle runs, description of the sample)."""
    import inputs
    base = wl_name[:-len("-loaded")] if wl_name.endswith("-loaded") else wl_name
    if base in ORACLE_SAMPLE:
        name, kws = ORACLE_SAMPLE[base]
        for kw in kws:
            sp = inputs.make_problem(name, **kw)
            if sp.n_dofs / ORACLE_DOF_STEPS_PER_S <= seconds_per_step:
                break
        fl = WORKLOADS[wl_name][1].get("face_load")
        if fl is not None:
            sp = inputs.with_face_load(sp, fl[0], comp=fl[1])
        return sp, (f"{sp.n_dofs}-DOF version of {wl_name} (same material, element type, dt/h, tolerance and "
                    f"load; the oracle's DOF-steps/s scale about linearly with DOFs)")
    return prob, wl_name


def run_reference(args, prob, wl_name, precision):
    """FP64 CPU oracle on the host cores: W untimed + K timed steps of the same workload."""
    import numpy as np  # noqa: F401
    from oracle import propagator
    prob, what = _oracle_problem(prob, wl_name, 150.0 / (args.steps + args.warmup))
    P = propagator.Propagator.from_problem(prob)
    for _ in range(args.warmup):
        P.step(prob.dt, prob.tol)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        P.step(prob.dt, prob.tol)
    dt = time.perf_counter() - t0
    value = prob.n_dofs * args.steps / dt
    cores = os.cpu_count()
    sample = f"{args.steps} oracle time steps of {what} after {args.warmup} warm-up steps"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": wl_name, "dofs": prob.n_dofs, "dt": prob.dt, "tol": prob.tol,
                   "precision": "fp64", "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline(prob, wl_name, budget_s=15.0):
    """The oracle as it stands, timed on a bounded sample (whole steps until ~budget_s)."""
    from oracle import propagator
    prob, what = _oracle_problem(prob, wl_name)
    P = propagator.Propagator.from_problem(prob)
    P.step(prob.dt, prob.tol)  # first step builds caches; not timed
    n = 0
    t0 = time.perf_counter()
    while True:
        P.step(prob.dt, prob.tol)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 50:
            break
    return {"value": prob.n_dofs * n / el, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} oracle time steps of {what} (after one untimed step), numpy/scipy FP64"}


def served_measurement(n_requests, horizon_scale, dof_range, ragged_slots=48, compare=None):
    """The served mixed batch (Poisson arrivals of beams and blocks, half linear, half
    Neo-Hookean): the MIXED ragged batched form served in real time (p50/p99 step latency),
    then the same requests queued at once in that form and as plain FP64 one at a time (equal
    work: DOF-steps/s, energy error of each form, MIXED vs FP64 state and energy)."""
    import numpy as np
    import inputs
    from paper_2405_05213_gb300 import etp, serve
    mix = inputs.served_mix(n_requests, horizon_scale=horizon_scale, dof_range=dof_range)
    reqs = [serve.Request(k, arr, p, steps, precision=etp.ETP_PREC_MIXED) for k, (arr, p, steps) in enumerate(mix)]
    srv = serve.Server(slots=ragged_slots, ragged=True)
    live = serve.summarize(srv.run(reqs, realtime=True), srv.wall)
    srv.close()
    sub = reqs if compare is None else reqs[:compare]
    seq = serve.Server(slots=1, keep_state=True)
    rs = seq.run([serve.Request(r.rid, 0.0, r.problem, r.steps, etp.ETP_PREC_FP64) for r in sub], realtime=False)
    fp64 = serve.summarize(rs, seq.wall)
    seq.close()
    b = serve.Server(slots=ragged_slots, ragged=True, keep_state=True)
    rb = b.run([serve.Request(r.rid, 0.0, r.problem, r.steps, etp.ETP_PREC_MIXED) for r in sub], realtime=False)
    mixed = serve.summarize(rb, b.wall)
    b.close()
    ok = [k for k in rs if rs[k].status == "ok" and k in rb and rb[k].status == "ok"]
    e_diff = max(abs(rb[k].energy - rs[k].energy) / abs(rs[k].energy0) for k in ok)
    u_diff = max(np.linalg.norm(rb[k].u - rs[k].u) / max(np.linalg.norm(rs[k].u), 1e-300) for k in ok)

    def drift(res, kind):
        v = [abs(res[k].energy - res[k].energy0) / res[k].energy0 for k in ok
             if (res[k].energy0 > 0 and (sub[k].problem.material == kind))]
        return float(max(v)) if v else None
    return {
        "requests": n_requests, "dofs": f"{dof_range[0]}-{dof_range[1]} log-uniform",
        "horizon_scale": horizon_scale, "poisson_rate_hz": 50.0, "tol": 1e-8,
        "served_realtime_mixed_ragged": {k: live[k] for k in ("dof_steps_per_s", "p50_step_ms", "p99_step_ms",
                                                              "wall_s", "failed")},
        "equal_work": {
            "requests": len(sub),
            "mixed_ragged_dof_steps_per_s": mixed["dof_steps_per_s"],
            "fp64_one_at_a_time_dof_steps_per_s": fp64["dof_steps_per_s"],
            "speedup_vs_fp64_one_at_a_time": mixed["dof_steps_per_s"] / fp64["dof_steps_per_s"],
            "p50_p99_step_ms_mixed_ragged": [mixed["p50_step_ms"], mixed["p99_step_ms"]],
            "p50_p99_step_ms_fp64_one_at_a_time": [fp64["p50_step_ms"], fp64["p99_step_ms"]],
            # energy error of each form: |E_end - E_0| / E_0 per request (the propagator's own
            # energy error, nonlinear members O(dt^2), linear members ~tol), max over requests
            "energy_error_linear": {"mixed": drift(rb, inputs.MAT_LINEAR), "fp64": drift(rs, inputs.MAT_LINEAR)},
            "energy_error_neohooke": {"mixed": drift(rb, inputs.MAT_NEOHOOKE),
                                      "fp64": drift(rs, inputs.MAT_NEOHOOKE)},
            # what the MIXED form adds: its final energy against the FP64 form's, relative to E_0
            "max_rel_energy_diff_mixed_vs_fp64": float(e_diff),
            "max_rel_u_diff_mixed_vs_fp64": float(u_diff),
            "failed": mixed["failed"] + fp64["failed"],
        },
    }


def run_serve(args):
    """Served mixed batch: Poisson arrivals of beams and blocks, continuous batching
    (MIXED precision) against plain FP64 one request at a time. Two batching forms:
    'ragged' (all admitted trajectories advance together, one etp_step_batch round at a
    time, shared launches) and 'streams' (worker threads, one CUDA stream per request)."""
    import inputs
    from paper_2405_05213_gb300 import etp, serve
    import __graft_entry__
    __graft_entry__.build()
    import numpy as np
    lo, hi = (int(x) for x in args.serve_dofs.split(","))
    mix = inputs.served_mix(args.serve_requests, horizon_scale=args.serve_horizon_scale, dof_range=(lo, hi))
    reqs = [serve.Request(k, arr, p, steps, precision=etp.ETP_PREC_MIXED) for k, (arr, p, steps) in enumerate(mix)]
    modes = ["ragged", "streams"] if args.serve_mode == "both" else [args.serve_mode]
    slots = {"ragged": args.serve_ragged_slots, "streams": args.serve_slots}

    def server(mode, **kw):
        return serve.Server(slots=slots[mode], ragged=(mode == "ragged"), **kw)

    served = {}
    for mode in modes:
        srv = server(mode)
        res = srv.run(reqs, realtime=True)
        served[mode] = serve.summarize(res, srv.wall)
        srv.close()
    # the same first requests, every way, for an equal-work comparison
    sub = reqs[: args.serve_compare]
    eq = {"requests": len(sub)}
    seq = serve.Server(slots=1, keep_state=True)
    rs = seq.run([serve.Request(r.rid, 0.0, r.problem, r.steps, etp.ETP_PREC_FP64) for r in sub], realtime=False)
    eq["fp64_one_at_a_time"] = serve.summarize(rs, seq.wall)
    for mode in modes:
        b = server(mode, keep_state=True)
        rb = b.run([serve.Request(r.rid, 0.0, r.problem, r.steps, etp.ETP_PREC_MIXED) for r in sub], realtime=False)
        e_diff = max(abs(rb[k].energy - rs[k].energy) / abs(rs[k].energy) for k in rs)
        u_diff = max(np.linalg.norm(rb[k].u - rs[k].u) / max(np.linalg.norm(rs[k].u), 1e-300) for k in rs)
        d = serve.summarize(rb, b.wall)
        d["max_rel_energy_diff_vs_fp64"] = float(e_diff)
        d["max_rel_u_diff_vs_fp64"] = float(u_diff)
        d["speedup_vs_fp64_one_at_a_time"] = d["dof_steps_per_s"] / eq["fp64_one_at_a_time"]["dof_steps_per_s"]
        eq[f"mixed_{mode}"] = d
        b.close()
    out = {
        "mode": "served-mix", "metric": METRIC, "unit": UNIT,
        "config": {"requests": args.serve_requests, "poisson_rate_hz": 50.0, "dofs": f"{lo}-{hi} log-uniform",
                   "horizon_scale": args.serve_horizon_scale, "slots": slots,
                   "materials": "50% linear / 50% Neo-Hookean", "tol": 1e-8},
        "served_realtime_mixed": served,
        "equal_work_subset": eq,
    }
    print(json.dumps(out), flush=True)


def _newmark_case(etp, p, T, target, max_steps, ep_grid, ref_steps):
    """Time to a relative L2 error target at horizon T for the propagator (steps x tolerance grid)
    and Newmark-beta (step halving from 10 steps), both FP64 on this GPU; the reference is the
    propagator at tol 1e-12 with ref_steps steps (its own error estimated against half as many)."""
    import numpy as np
    import torch
    stream = torch.cuda.Stream()  # a created stream: the Newmark CG blocks run as captured graphs
    ctx = etp.Context(0, stream=stream.cuda_stream)
    mesh = etp.Mesh.from_problem(ctx, p)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    def run(fn, n):
        t = etp.Trajectory(mesh, p.u0, p.v0, etp.ETP_PREC_FP64, 256)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            fn(t, T / n)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        u, v = t.state()
        t.close()
        return sec, u, v

    ep_step = lambda tol: (lambda t, dt: t.step(dt, tol))
    nm_step = lambda t, dt: etp.etp_newmark_step(t.h, dt, 1e-12)
    for fn in (ep_step(1e-8), nm_step):  # warm-up of both paths (first-use set-up)
        try:
            run(fn, 40)
        except etp.EtpError:
            pass
    _, u_ref, v_ref = run(ep_step(1e-12), ref_steps)
    _, u_h, v_h = run(ep_step(1e-12), ref_steps // 2)
    ep = []
    for n in ep_grid:
        for tol in (1e-5, 1e-7, 1e-9):
            try:
                sec, u, v = run(ep_step(tol), n)
            except etp.EtpError:  # a step larger than m_cap = 256 allows
                continue
            ep.append({"steps": n, "dt": T / n, "tol": tol, "s": sec, "err_u": rel(u, u_ref), "err_v": rel(v, v_ref)})
    nm = []
    n = 10
    while n <= max_steps:
        try:
            sec, u, v = run(nm_step, n)
        except etp.EtpError:
            n *= 2
            continue
        nm.append({"steps": n, "dt": T / n, "s": sec, "err_u": rel(u, u_ref), "err_v": rel(v, v_ref)})
        if nm[-1]["err_u"] <= target and nm[-1]["err_v"] <= target:
            break
        n *= 2
    out = {"workload": f"{p.name}-{p.n_dofs}dof", "dofs": p.n_dofs, "horizon": T, "target_rel_err": target,
           "reference": f"propagator, tol 1e-12, {ref_steps} steps",
           "reference_err_est": {"u": rel(u_h, u_ref) / 3.0, "v": rel(v_h, v_ref) / 3.0},
           "ep_runs": ep, "newmark_runs": nm}
    for q in ("u", "v"):
        e_ok = [r for r in ep if r["err_" + q] <= target]
        n_ok = [r for r in nm if r["err_" + q] <= target]
        best_e = min(e_ok, key=lambda r: r["s"]) if e_ok else None
        best_n = min(n_ok, key=lambda r: r["s"]) if n_ok else None
        out["target_" + q] = {"propagator": best_e, "newmark": best_n,
                              "speedup": (best_n["s"] / best_e["s"]) if best_e and best_n else None}
    mesh.close()
    ctx.close()
    return out


def run_newmark(args):
    """Same-box comparison with the paper's comparison integrator (Section 6): on a struck beam
    (broadband initial velocity), linear, Saint Venant-Kirchhoff and Yeoh, the wall time each method needs
    to reach a relative error target in u and in v at a fixed horizon, both on this GPU in FP64:
    the exponential propagator (steps x tolerance grid) and average-acceleration Newmark-beta
    (step halving; Newton with the consistent tangent for the nonlinear materials)."""
    import dataclasses
    import inputs
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp
    nel = tuple(int(x) for x in args.newmark_nel.split(","))
    T, target = args.newmark_horizon, args.newmark_target
    lin = inputs.beam_linear_impulse(nel=nel)
    out = {"mode": "newmark-comparison", "precision": "f64",
           "linear": _newmark_case(etp, lin, T, target, args.newmark_max_steps, (5, 10, 20, 40, 80), 200)}
    # SVK with the linear beam's small-strain moduli, struck 5x harder (finite strains; harder
    # strikes compress the beam into the range where the SVK tangent loses definiteness)
    E, nu = lin.params
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    svk = dataclasses.replace(lin, name="beam-svk-impulse-q1", material=inputs.MAT_SVK, params=(lam, mu),
                              v0=5.0 * lin.v0)
    out["svk"] = _newmark_case(etp, svk, T, target, args.newmark_max_steps, (10, 20, 40, 80, 160), 800)
    # Yeoh with the paper's Treloar rubber constants (Section 6.3: C10 = 100, C20 = -1, C30 = 0.01,
    # D1 = 0.001), struck as hard as the SVK beam; Newmark's Newton iterations use the exact tangent
    yeoh = dataclasses.replace(lin, name="beam-yeoh-impulse-q1", material=inputs.MAT_YEOH,
                               params=(100.0, -1.0, 0.01, 0.001), v0=5.0 * lin.v0)
    out["yeoh"] = _newmark_case(etp, yeoh, T, target, args.newmark_max_steps, (10, 20, 40, 80, 160), 800)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--serve", action="store_true", help="served mixed-batch measurement (separate JSON line)")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-horizon-scale", type=float, default=0.05)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-ragged-slots", type=int, default=48)
    ap.add_argument("--serve-mode", default="both", choices=["both", "ragged", "streams"])
    ap.add_argument("--serve-dofs", default="2000,500000", help="DOF range of the served requests (lo,hi)")
    ap.add_argument("--newmark", action="store_true", help="same-box comparison with Newmark-beta (separate JSON line)")
    ap.add_argument("--newmark-nel", default="80,8,8")
    ap.add_argument("--newmark-horizon", type=float, default=1.0)
    ap.add_argument("--newmark-target", type=float, default=1e-4)
    ap.add_argument("--newmark-max-steps", type=int, default=20480)
    ap.add_argument("--serve-compare", type=int, default=24)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="etp", choices=["etp", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="built-in launch shapes instead of autotuned ones")
    ap.add_argument("--krylov", default="arnoldi", choices=["arnoldi", "lanczos"],
                    help="Krylov process (lanczos: energy inner product, linear materials)")
    ap.add_argument("--profile-steps", type=int, default=3,
                    help="steps of the separate per-kernel-class event-profiled pass")
    ap.add_argument("--no-serve", action="store_true", help="skip the served mixed-batch object of the line")
    ap.add_argument("--served-requests", type=int, default=48)
    ap.add_argument("--served-horizon-scale", type=float, default=0.1)
    ap.add_argument("--served-dofs", default="2000,100000")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.serve:
        run_serve(args)
        return
    if args.newmark:
        run_newmark(args)
        return

    prob, precision = make_workload_problem(args.workload)
    import inputs as inputs_mod
    from paper_2405_05213_gb300 import replicas
    ws, rank, local = replicas.dist_env()

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, prob, args.workload, precision)), flush=True)
        return

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    replicas.init("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp

    ctx = etp.Context(local)
    stream = torch.cuda.current_stream(local)
    prec = etp.ETP_PREC_MIXED if precision == "mixed" else etp.ETP_PREC_FP64
    mesh = etp.Mesh.from_problem(ctx, prob)
    traj = etp.Trajectory(mesh, prob.u0, prob.v0, prec, prob.m_cap)
    if prob.load is not None:
        traj.set_load(prob.load)
    if args.krylov == "lanczos":
        traj.set_krylov(etp.ETP_KRYLOV_LANCZOS_ENERGY)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    # launch shapes picked by the library's autotuner (untimed set-up)
    t_tune = time.perf_counter()
    n_tuned = 0 if args.no_autotune else etp.etp_autotune(traj.h, 3)
    t_tune = time.perf_counter() - t_tune

    def barrier():
        replicas.barrier()
        torch.cuda.synchronize()

    # the clock sampler starts before the warm-up: nvidia-smi's start-up (a few tens of ms of
    # driver queries) stalls the GPU work of a short timed region if it falls inside it
    clk = ClockSampler(local).__enter__()
    time.sleep(0.5)
    for _ in range(args.warmup):
        traj.step(prob.dt, prob.tol)
    ms_list, m_list = [], []
    launches0 = etp.etp_launch_count(ctx.h)
    barrier()
    try:
        for _ in range(args.steps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m, _ = traj.step(prob.dt, prob.tol)
            b.record(stream)
            b.synchronize()
            ms_list.append(a.elapsed_time(b))
            m_list.append(m)
        barrier()
    finally:
        clk.__exit__(None, None, None)
    launches = etp.etp_launch_count(ctx.h) - launches0
    total_ms = replicas.max_over_ranks(sum(ms_list), device=f"cuda:{local}")
    value = replicas.aggregate_throughput(prob.n_dofs * args.steps, total_ms * 1e-3, ws)

    # per-kernel-class breakdown from a separate pass with event profiling on (the
    # timed steps above run without it): CUDA events around every launch, on the
    # library's stream, L2 flushed between steps as above
    etp.etp_profile_reset(ctx.h)
    etp.etp_profile_enable(ctx.h, True)
    prof_ms = 0.0
    for _ in range(args.profile_steps):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        traj.step(prob.dt, prob.tol)
        b.record(stream)
        b.synchronize()
        prof_ms += a.elapsed_time(b)
    etp.etp_profile_enable(ctx.h, False)
    prof = etp.etp_profile_read(ctx.h)
    prof_total = max(prof_ms, 1e-9)

    # Roofline of the dominant kernel class. Algorithmic bytes per launch: the operator apply's
    # B_apply = 2 N_f s + N_f s_u + 4 n_e (x read, z written, the frozen displacement, the element
    # scale) for the element pass; each Gram-Schmidt pass reads every basis column it uses once
    # (and writes its outputs); the state combine reads the m-1 basis columns and the state. The
    # element pass also has an algorithmic flop count (the secant-stress contractions per Gauss
    # point). Each class is reported against the resource it comes closest to saturating: HBM
    # (measured copy bandwidth) or the FP32 pipe (derived from unit counts and clock).
    peak, peak_kind = _peaks()
    fpeak = _fp32_peak_tflops()
    s_k = 4 if precision == "mixed" else 8
    n_free = prob.n_dofs - len(prob.fixed_dofs)
    b_apply = 2 * n_free * s_k + (n_free * s_k if prob.material != inputs_mod.MAT_LINEAR else 0) + \
        (4 * prob.mesh.n_elems if prob.elem_scale is not None else 0)
    model_classes = ("cgs_dot", "cgs_update_dot", "cgs_update_norm", "fused_arnoldi_step", "node_gather",
                     "state_combine", "frozen_build", "lanczos")
    by_kernel = {}
    for k, v in prof.items():
        if v["launches"] == 0:
            continue
        e = {"launches": v["launches"], "ms": round(v["ms"], 4), "share_of_step": round(v["ms"] / prof_total, 4)}
        if v["ms"] > 0:
            if k == "elem_apply":
                gbs = b_apply * v["launches"] / 1e9 / (v["ms"] / 1e3)
                e["algorithmic_GBps"] = round(gbs, 1)
                e["frac_of_measured_hbm"] = round(gbs / peak, 4)
                e["streamed_GBps_model"] = round((v["bytes"] / 1e9) / (v["ms"] / 1e3), 1)
            elif v["bytes"] > 0:
                gbs = (v["bytes"] / 1e9) / (v["ms"] / 1e3)
                e["GBps"] = round(gbs, 1)
                if k in model_classes:
                    e["frac_of_measured_hbm"] = round(gbs / peak, 4)
            if v.get("flops", 0) > 0:
                tf = (v["flops"] / 1e12) / (v["ms"] / 1e3)
                e["TFLOPs"] = round(tf, 2)
                e["frac_of_fp32_peak"] = round(tf / fpeak, 4)
        by_kernel[k] = e
    dom = max((k for k in by_kernel if k != "other"), key=lambda k: prof[k]["ms"])
    d = prof[dom]
    nl = max(d["launches"], 1)
    e = by_kernel[dom]
    hbm_frac = e.get("frac_of_measured_hbm", 0.0)
    alu_frac = e.get("frac_of_fp32_peak", 0.0)
    alg_bytes = b_apply if dom == "elem_apply" else d["bytes"] / nl
    if alu_frac > hbm_frac:
        achieved = (d["flops"] / 1e12) / (d["ms"] / 1e3)
        roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fpeak, "unit": "TFLOP/s",
                    "frac": achieved / fpeak,
                    "peak_source": "derived: SMs x 128 FP32 lanes x 2 flop/FMA x max SM clock",
                    "algorithmic_flops_per_launch": d["flops"] / nl,
                    "hbm_frac_on_algorithmic_bytes": hbm_frac}
    else:
        achieved = alg_bytes * nl / 1e9 / (d["ms"] / 1e3)
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": peak_kind, "fp32_frac": alu_frac}
    roofline.update({"traffic": _traffic(dom, args.workload), "algorithmic_bytes_per_launch": alg_bytes,
                     "avg_launch_us": 1e3 * d["ms"] / nl, "share_of_step": d["ms"] / prof_total,
                     "profiled_steps": args.profile_steps, "by_kernel": by_kernel})

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        n = prob.n_dofs
        hu = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        hv = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        etp.etp_state_get_into(traj.h, hu, hv)
        barrier()
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            etp.etp_state_upload(traj.h, hu, hv)
            traj.step(prob.dt, prob.tol)
            etp.etp_state_get_into(traj.h, hu, hv)
            b.record(stream)
            b.synchronize()
            e2e_ms += a.elapsed_time(b)
        e2e_ms = replicas.max_over_ranks(e2e_ms, device=f"cuda:{local}")
        e2e = {"value": replicas.aggregate_throughput(n * args.steps, e2e_ms * 1e-3, ws), "unit": UNIT,
               "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 2 * 8 * n}

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64" if precision == "mixed" else "f64",
        "data": "synthetic (seeded generators in inputs/)",
        "config": {"workload": args.workload, "dofs": prob.n_dofs, "dt": prob.dt, "tol": prob.tol,
                   "precision": precision, "krylov": args.krylov, "m_per_step_corrector": [int(x) for x in m_list],
                   "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{ws}",
                   "autotuned_shapes": int(n_tuned), "autotune_s": round(t_tune, 2)},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if not args.no_serve and ws == 1:
        lo, hi = (int(x) for x in args.served_dofs.split(","))
        out["served"] = served_measurement(args.served_requests, args.served_horizon_scale, (lo, hi))
    if not args.no_cpu_baseline and ws == 1 and (args.workload in ORACLE_SAMPLE or prob.n_dofs <= 200000):
        out["cpu_baseline"] = cpu_baseline(prob, args.workload)
    print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
