"""Continuous-batching server for propagation requests (served mixed batch workload).

Requests (a mesh, a material, an initial state, dt, a horizon and a tolerance)
arrive over time. The server admits a queued request as soon as a slot is free
and its device-memory need (the library's exact count) fits the budget, and
hands its trajectory to the
native batch of libetp (``etp_batch_*``): worker threads in the library step
every admitted trajectory, each on its own CUDA stream, so the kernels of
different trajectories overlap on the GPU; the library retires a trajectory
when its horizon is done (or its step fails) and releases its share of the
budget. With ``ragged=True`` the requests instead go to a few size-class
contexts ("lanes", one CUDA stream each) and the library's ragged batch runs
one engine per lane: each tick advances every active Krylov solve of the lane
by one Arnoldi step in shared launches (one element-pass launch per class, one
persistent-step launch), and the lanes' kernels overlap on the GPU, so small
requests do not wait for the ticks of large ones. The largest requests, whose
steps fill the GPU alone, get a context and engine of their own.
This module only creates the per-request objects, feeds arrivals and
collects results; every numerical step runs in libetp.
"""
from __future__ import annotations

import heapq
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


def footprint(problem, precision, m_cap, device=0):
    """Exact device bytes of one request (trajectory + mesh), from the library's own count."""
    ctx = etp.Context(device)
    mesh = etp.Mesh.from_problem(ctx, problem)
    try:
        tb, mb = etp.etp_traj_footprint(mesh.h, precision, m_cap)
    finally:
        mesh.close()
        ctx.close()
    return tb + mb


class Server:
    """Admit, run and retire propagation requests with at most `slots` concurrent trajectories."""

    # ragged mode: requests of fewer DOFs than edge k go to lane k (the last lane takes the rest
    # below SOLO_DOFS); requests of SOLO_DOFS or more, whose Arnoldi steps fill the GPU by
    # themselves, get a context (stream and engine) of their own
    LANE_EDGES = (8000, 30000, 80000)
    SOLO_DOFS = 150000

    def __init__(self, device=0, slots=8, memory_budget=None, keep_state=False, ragged=False, lanes=None):
        import torch
        self.device = device
        self.slots = slots
        free, total = torch.cuda.mem_get_info(device)
        self.budget = int(memory_budget if memory_budget is not None else 0.8 * free)
        self.keep_state = keep_state
        self.results = {}
        self.rejected = []
        self.peak_reserved = 0  # largest budget share in use at once (library count)
        self.ragged = ragged
        self._lanes = []
        if ragged:
            edges = self.LANE_EDGES if lanes is None else tuple(lanes)
            self._edges = edges
            for _ in range(len(edges) + 1):
                st = torch.cuda.Stream(device=device)
                self._lanes.append((st, etp.Context(device, stream=st.cuda_stream)))
            self._ctx = self._lanes[0][1]
            self._batch = etp.etp_batch_create_ragged(self._ctx.h, self.budget)
        else:
            self._ctx = etp.Context(device)
            self._batch = etp.etp_batch_create(self._ctx.h, self.budget, max(1, slots))

    def close(self):
        if self._batch:
            etp.etp_batch_destroy(self._batch)
            self._batch = None
        if self._lanes:
            for _, ctx in self._lanes:
                ctx.close()
            self._lanes = []
        elif self._ctx is not None:
            self._ctx.close()
        self._ctx = None

    def _lane(self, n_dofs):
        """Context of the size class of a request of n_dofs DOFs (ragged mode)."""
        k = sum(1 for e in self._edges if n_dofs >= e)
        return self._lanes[k][1]

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stage(self, req):
        """Create the request's context (own stream; its lane's in ragged mode) and mesh; the
        exact footprint decides admission."""
        import torch
        if self.ragged and req.problem.n_dofs < self.SOLO_DOFS:
            stream, ctx = None, None
            mesh = etp.Mesh.from_problem(self._lane(req.problem.n_dofs), req.problem)
        else:
            stream = torch.cuda.Stream(device=self.device)
            ctx = etp.Context(self.device, stream=stream.cuda_stream)
            mesh = etp.Mesh.from_problem(ctx, req.problem)
        tb, mb = etp.etp_traj_footprint(mesh.h, req.precision, req.m_cap)
        return {"req": req, "stream": stream, "ctx": ctx, "mesh": mesh, "traj": None, "need": tb + mb}

    def _open(self, obj, t_start):
        """Create the trajectory of a staged request."""
        req = obj["req"]
        obj["traj"] = etp.Trajectory(obj["mesh"], req.problem.u0, req.problem.v0, req.precision, req.m_cap)
        res = Result(req.rid, req.problem.n_dofs, 0, time.perf_counter() - t_start, 0.0)
        res.energy0 = obj["traj"].energy()[0]
        obj["res"] = res

    @staticmethod
    def _close(live):
        if live["traj"] is not None:
            live["traj"].close()
        live["mesh"].close()
        if live["ctx"] is not None:
            live["ctx"].close()

    def _retire(self, live, status, t_start):
        res, traj = live["res"], live["traj"]
        steps, _, _, ms = etp.etp_batch_traj_info(self._batch, traj.h)
        res.steps_done = steps
        res.step_latency_ms = [float(x) for x in ms]
        if status != etp.ETP_OK:
            res.status = f"error: status {status}"
        try:
            res.energy = traj.energy()[0]
            if self.keep_state:
                res.u, res.v = traj.state()
        except etp.EtpError as e:
            res.status = f"error: {e}"
        etp.etp_batch_forget(self._batch, traj.h)
        self._close(live)
        res.finished = time.perf_counter() - t_start
        self.results[res.rid] = res

    def run(self, requests, realtime=True):
        """Serve `requests` (by arrival time); returns the results by request id."""
        queue = []
        for r in requests:
            heapq.heappush(queue, (r.arrival, r.rid, r))
        t_start = time.perf_counter()
        pending = []  # arrived, waiting for a slot or memory (FIFO)
        live = {}     # trajectory handle value -> request objects
        staged = None  # head-of-line request with its context and mesh already created
        while queue or pending or live:
            now = time.perf_counter() - t_start
            while queue and (not realtime or queue[0][0] <= now):
                pending.append(heapq.heappop(queue)[2])
            reserved, _ = etp.etp_batch_usage(self._batch)
            while pending and len(live) < self.slots:
                req = pending[0]
                try:
                    if staged is None or staged["req"] is not req:
                        staged = self._stage(req)
                    if staged["need"] > self.budget:  # never fits: reject
                        self.rejected.append(req.rid)
                        self._close(staged)
                        staged = None
                        pending.pop(0)
                        continue
                    if reserved + staged["need"] > self.budget:
                        break  # wait for a retirement
                    self._open(staged, t_start)
                except etp.EtpError as e:
                    if staged is not None:
                        self._close(staged)
                        staged = None
                    pending.pop(0)
                    self.results[req.rid] = Result(req.rid, req.problem.n_dofs, 0, now, now, status=f"error: {e}")
                    continue
                p = req.problem
                if not etp.etp_batch_admit(self._batch, staged["traj"].h, req.steps, p.dt, p.tol):
                    # the library's count disagrees with ours: not now, or never if nothing is running
                    staged["traj"].close()
                    staged["traj"] = None
                    if not live:
                        self.rejected.append(req.rid)
                        self._close(staged)
                        staged = None
                        pending.pop(0)
                        continue
                    break
                pending.pop(0)
                live[staged["traj"].h.value] = staged
                staged = None
                reserved, _ = etp.etp_batch_usage(self._batch)
                self.peak_reserved = max(self.peak_reserved, reserved)
            if live:
                etp.etp_batch_tick(self._batch)
                for th, status in etp.etp_batch_retired(self._batch):
                    self._retire(live.pop(th), status, t_start)
            elif queue and realtime:
                time.sleep(max(0.0, min(0.05, queue[0][0] - (time.perf_counter() - t_start))))
        if staged is not None:
            self._close(staged)
        self.wall = time.perf_counter() - t_start
        return self.results


def summarize(results, wall):
    lat = [np.asarray(r.step_latency_ms) for r in results.values() if r.step_latency_ms]
    lat = np.concatenate(lat) if lat else np.zeros(0)
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
