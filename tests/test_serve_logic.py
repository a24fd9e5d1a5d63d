"""Admission and retirement logic of serve.Server on the CPU, against a fake library
with the contract of include/etp.h's etp_batch_* calls (no GPU)."""
import types

import numpy as np
import pytest

import inputs


class _H:
    _next = 1

    def __init__(self):
        self.value = _H._next
        _H._next += 1


def _fake_etp(fail_rids=(), exact_extra=0):
    ns = types.SimpleNamespace()
    ns.ETP_OK, ns.ETP_ERR_OOM, ns.ETP_ERR_NOT_CONVERGED = 0, 2, 4
    ns.ETP_PREC_FP64, ns.ETP_PREC_MIXED = 0, 1

    class EtpError(RuntimeError):
        pass
    ns.EtpError = EtpError

    class Context:
        def __init__(self, device=0, stream=None):
            self.h = _H()

        def close(self):
            pass

    class Mesh:
        @classmethod
        def from_problem(cls, ctx, prob):
            m = cls()
            m.h, m.prob = _H(), prob
            return m

        def close(self):
            pass

    trajs = {}

    class Trajectory:
        def __init__(self, mesh, u0, v0, precision, m_cap):
            self.h, self.mesh, self.n = _H(), mesh, mesh.prob.n_dofs
            trajs[self.h.value] = self

        def energy(self):
            return (1.0, 0.5, 0.5)

        def state(self):
            return np.zeros(self.n), np.zeros(self.n)

        def close(self):
            pass
    ns.Context, ns.Mesh, ns.Trajectory = Context, Mesh, Trajectory

    def footprint(mesh_h, precision, m_cap):
        return 100 * 1000 + 0 * m_cap, 1000  # every request: 101,000 bytes
    ns.etp_traj_footprint = footprint

    class Batch:
        def __init__(self, budget):
            self.budget, self.active, self.retired, self.info = budget, {}, [], {}

    def create(ctx_h, budget, workers):
        return Batch(budget)

    def admit(b, th, n_steps, dt, tol):
        need = 101_000 + exact_extra
        if sum(a["need"] for a in b.active.values()) + need > b.budget:
            return False
        b.active[th.value] = {"need": need, "left": n_steps}
        b.info[th.value] = [0, 0, False, []]
        return True

    def tick(b):
        done = 0
        for k, a in list(b.active.items()):
            t = trajs[k]
            rid = t.mesh.prob.notes.get("rid")
            inf = b.info[k]
            inf[3].append(1.0)
            if rid in fail_rids:
                inf[1] = ns.ETP_ERR_NOT_CONVERGED
            else:
                inf[0] += 1
                a["left"] -= 1
                done += 1
            if a["left"] == 0 or inf[1]:
                inf[2] = True
                b.retired.append((k, inf[1]))
                del b.active[k]
        return done

    def retired(b, max_n=256):
        out, b.retired = b.retired, []
        return out

    def traj_info(b, th):
        sd, st, rt, ms = b.info[th.value]
        return sd, st, rt, np.asarray(ms, dtype=np.float32)

    def usage(b):
        return sum(a["need"] for a in b.active.values()), len(b.active)
    ns.etp_batch_create, ns.etp_batch_admit, ns.etp_batch_tick = create, admit, tick
    ns.etp_batch_retired, ns.etp_batch_traj_info, ns.etp_batch_usage = retired, traj_info, usage
    ns.etp_batch_forget = lambda b, th: b.info.pop(th.value)
    ns.etp_batch_destroy = lambda b: None
    return ns


@pytest.fixture
def fake_server(monkeypatch):
    import torch
    from paper_2405_05213_gb300 import serve
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda d=0: (1 << 30, 1 << 31))
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=0: types.SimpleNamespace(cuda_stream=0))

    def make(fail_rids=(), exact_extra=0, **kw):
        monkeypatch.setattr(serve, "etp", _fake_etp(fail_rids, exact_extra))
        return serve, serve.Server(**kw)
    return make


def _requests(serve, n, steps=3):
    mix = inputs.served_mix(n, dof_range=(2000, 4000), horizon=(2, 3))
    reqs = []
    for k, (arr, p, _) in enumerate(mix):
        p.notes["rid"] = k
        reqs.append(serve.Request(k, 0.0, p, steps))
    return reqs


def test_budget_limits_concurrency_and_all_complete(fake_server):
    serve, srv = fake_server(slots=4, memory_budget=250_000)
    res = srv.run(_requests(serve, 6), realtime=False)
    assert len(res) == 6 and all(r.status == "ok" and r.steps_done == 3 for r in res.values())
    assert srv.peak_reserved == 2 * 101_000  # two fit in 250,000, never three
    assert all(len(r.step_latency_ms) == 3 for r in res.values())


def test_failed_request_retires_alone(fake_server):
    serve, srv = fake_server(fail_rids={1}, slots=3, memory_budget=10**9)
    res = srv.run(_requests(serve, 4), realtime=False)
    assert res[1].status.startswith("error") and res[1].steps_done == 0
    assert all(res[k].status == "ok" and res[k].steps_done == 3 for k in (0, 2, 3))


def test_oversize_and_disagreeing_counts_are_rejected_not_retried(fake_server):
    serve, srv = fake_server(slots=2, memory_budget=100_000)  # below one request's footprint
    srv.run(_requests(serve, 2), realtime=False)
    assert srv.rejected == [0, 1] and srv.results == {}
    # the library's exact count is above the server's: with nothing running, reject instead of looping
    serve, srv = fake_server(exact_extra=10**6, slots=2, memory_budget=200_000)
    srv.run(_requests(serve, 2), realtime=False)
    assert srv.rejected == [0, 1]
