"""Continuous-batching server for propagation requests (served mixed batch workload).

Requests (a mesh, a material, an initial state, dt, a horizon and a tolerance)
arrive over time. The server admits a queued request as soon as a slot is free
and its device-memory need fits the budget, keeps each admitted trajectory's
state and Krylov workspace resident on the device, and steps all admitted
trajectories concurrently: each slot is a host worker thread driving its own
CUDA stream through the C ABI (ctypes releases the GIL during library calls),
so the kernels of different trajectories overlap on the GPU. A finished
trajectory frees its slot and memory, and the next request is admitted.

Every numerical step runs in libetp; this module only schedules.
"""
from __future__ import annotations

import heapq
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import etp


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the server start
    problem: object         # inputs.Problem
    steps: int
    precision: int = etp.ETP_PREC_MIXED
    m_cap: int = 64


@dataclass
class Result:
    rid: int
    dofs: int
    steps_done: int
    admitted: float
    finished: float
    step_latency_ms: list = field(default_factory=list)
    energy0: float = 0.0
    energy: float = 0.0
    u: np.ndarray | None = None
    v: np.ndarray | None = None
    status: str = "ok"


def device_bytes_needed(prob, precision, m_cap):
    """Device memory of one trajectory plus its mesh (what admission reserves)."""
    n_nodes = prob.mesh.n_nodes
    nn_pad = -(-n_nodes // 128) * 128
    L = 6 * nn_pad
    s = 8 if precision == etp.ETP_PREC_FP64 else 4
    nen = prob.mesh.conn.shape[1]
    ne = prob.mesh.n_elems
    basis = (m_cap + 1) * L * s
    vectors = 2 * L * 8 + L * s + 3 * 3 * nn_pad * s
    elem = ne * nen * 3 * s + ne * nen * 4 * 2 + n_nodes * 4
    geo = ne * nen * 10 * 12  # general-geometry tables (boxes skip them: reserved conservatively)
    small = (m_cap + 1) * m_cap * 8 + 8 * 6 * m_cap * m_cap * 8 + (1 << 20)
    # stored frozen coefficients of two states (fields per Gauss point by material)
    nf = {etp.ETP_MAT_LINEAR: 0, etp.ETP_MAT_SVK: 9, etp.ETP_MAT_NEOHOOKE: 25,
          etp.ETP_MAT_MOONEY_RIVLIN: 33}.get(prob.material, 26)
    frozen = 2 * nf * ne * nen * s
    return basis + vectors + elem + geo + small + frozen + 3 * nn_pad * 8 * 3


class Server:
    """Admit, run and retire propagation requests with `slots` concurrent trajectories."""

    def __init__(self, device=0, slots=8, memory_budget=None, keep_state=False):
        import torch
        self.device = device
        self.slots = slots
        free, total = torch.cuda.mem_get_info(device)
        self.budget = int(memory_budget if memory_budget is not None else 0.8 * free)
        self.keep_state = keep_state
        self._lock = threading.Lock()
        self._cv = threading.Condition(self._lock)
        self._reserved = 0
        self._active = 0
        self.results = {}
        self.rejected = []

    def _fits(self, need):
        return self._active < self.slots and self._reserved + need <= self.budget

    def _run_one(self, req, need, t_start):
        import torch
        res = Result(req.rid, req.problem.n_dofs, 0, time.perf_counter() - t_start, 0.0)
        try:
            stream = torch.cuda.Stream(device=self.device)
            ctx = etp.Context(self.device, stream=stream.cuda_stream)
            mesh = etp.Mesh.from_problem(ctx, req.problem)
            traj = etp.Trajectory(mesh, req.problem.u0, req.problem.v0, req.precision, req.m_cap)
            res.energy0 = traj.energy()[0]
            p = req.problem
            for _ in range(req.steps):
                t0 = time.perf_counter()
                traj.step(p.dt, p.tol)
                res.step_latency_ms.append(1e3 * (time.perf_counter() - t0))
                res.steps_done += 1
            res.energy = traj.energy()[0]
            if self.keep_state:
                res.u, res.v = traj.state()
            traj.close()
            mesh.close()
            ctx.close()
        except Exception as e:  # the request fails alone; the server continues
            res.status = f"error: {e}"
        res.finished = time.perf_counter() - t_start
        with self._cv:
            self.results[req.rid] = res
            self._reserved -= need
            self._active -= 1
            self._cv.notify_all()

    def run(self, requests, realtime=True):
        """Serve `requests` (sorted by arrival); returns the results by request id."""
        queue = []
        for r in requests:
            heapq.heappush(queue, (r.arrival, r.rid, r))
        t_start = time.perf_counter()
        threads = []
        pending = []  # arrived, waiting for a slot or memory (FIFO)
        while queue or pending:
            now = time.perf_counter() - t_start
            while queue and (not realtime or queue[0][0] <= now):
                pending.append(heapq.heappop(queue)[2])
            with self._cv:
                while pending:
                    req = pending[0]
                    need = device_bytes_needed(req.problem, req.precision, req.m_cap)
                    if need > self.budget:
                        self.rejected.append(req.rid)
                        pending.pop(0)
                        continue
                    if not self._fits(need):
                        break
                    pending.pop(0)
                    self._reserved += need
                    self._active += 1
                    th = threading.Thread(target=self._run_one, args=(req, need, t_start), daemon=True)
                    th.start()
                    threads.append(th)
                if pending or (queue and realtime):
                    wait = 0.002
                    if queue and not pending:
                        wait = max(0.0, min(0.05, queue[0][0] - (time.perf_counter() - t_start)))
                    self._cv.wait(timeout=wait)
        for th in threads:
            th.join()
        self.wall = time.perf_counter() - t_start
        return self.results


def summarize(results, wall):
    lat = np.concatenate([np.asarray(r.step_latency_ms) for r in results.values() if r.step_latency_ms])
    dof_steps = sum(r.dofs * r.steps_done for r in results.values())
    errs = [abs(r.energy - r.energy0) / r.energy0 for r in results.values() if r.energy0 > 0]
    return {
        "requests": len(results),
        "failed": sum(1 for r in results.values() if r.status != "ok"),
        "dof_steps_per_s": dof_steps / wall,
        "wall_s": wall,
        "p50_step_ms": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_step_ms": float(np.percentile(lat, 99)) if lat.size else None,
        "max_rel_energy_drift": float(max(errs)) if errs else None,  # |E_end - E_0| / E_0 of each run
    }
