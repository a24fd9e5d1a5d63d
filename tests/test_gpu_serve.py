"""Served mixed batch (GPU): continuous batching gives each request the result it gets alone."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def test_results_identical_alone_and_in_the_mix():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp, serve
    mix = inputs.served_mix(6, dof_range=(2000, 40000), horizon=(4, 12))
    reqs = [serve.Request(k, 0.002 * k, p, steps) for k, (arr, p, steps) in enumerate(mix)]
    # in the mix: all admitted together, overlapping on the GPU
    mixed = serve.Server(slots=6, keep_state=True).run(reqs, realtime=False)
    # alone: one request at a time
    alone = {}
    for r in reqs:
        alone.update(serve.Server(slots=1, keep_state=True).run([r], realtime=False))
    for k in range(len(reqs)):
        a, b = alone[k], mixed[k]
        assert a.status == "ok" and b.status == "ok", (a.status, b.status)
        assert a.steps_done == b.steps_done == reqs[k].steps
        assert np.array_equal(a.u, b.u) and np.array_equal(a.v, b.v)
    s = serve.summarize(mixed, 1.0)
    assert s["failed"] == 0 and s["p99_step_ms"] >= s["p50_step_ms"] > 0


def test_ragged_server_results_identical_alone_and_in_the_mix():
    """Ragged mode: all admitted requests advance together (etp_step_batch rounds, shared launches,
    arrivals joining as others retire); each result is bitwise what the request gets alone."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import serve
    mix = inputs.served_mix(8, dof_range=(2000, 40000), horizon=(3, 9))
    reqs = [serve.Request(k, 0.001 * k, p, steps) for k, (arr, p, steps) in enumerate(mix)]
    srv = serve.Server(slots=5, ragged=True, keep_state=True)  # fewer slots than requests: arrivals join
    mixed = srv.run(reqs, realtime=False)
    srv.close()
    for r in reqs:
        alone = serve.Server(slots=1, keep_state=True).run([r], realtime=False)[r.rid]
        b = mixed[r.rid]
        assert alone.status == "ok" and b.status == "ok", (alone.status, b.status)
        assert b.steps_done == alone.steps_done == r.steps
        assert np.array_equal(alone.u, b.u) and np.array_equal(alone.v, b.v)
    s = serve.summarize(mixed, 1.0)
    assert s["failed"] == 0 and s["p99_step_ms"] >= s["p50_step_ms"] > 0


def test_admission_respects_memory_budget():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import serve
    mix = inputs.served_mix(4, dof_range=(2000, 8000), horizon=(2, 3))
    reqs = [serve.Request(k, 0.0, p, steps) for k, (arr, p, steps) in enumerate(mix)]
    need = max(serve.footprint(r.problem, r.precision, r.m_cap) for r in reqs)
    srv = serve.Server(slots=4, memory_budget=int(1.5 * need), keep_state=False)
    res = srv.run(reqs, realtime=False)
    assert len(res) == 4 and all(r.status == "ok" for r in res.values())
    assert 0 < srv.peak_reserved <= 1.5 * need
    big = serve.Server(slots=2, memory_budget=1024)
    big.run(reqs[:1], realtime=False)
    assert big.rejected == [0]


def _objects(prob, precision, m_cap=64):
    from paper_2405_05213_gb300 import etp
    import torch
    stream = torch.cuda.Stream()
    ctx = etp.Context(0, stream=stream.cuda_stream)
    mesh = etp.Mesh.from_problem(ctx, prob)
    traj = etp.Trajectory(mesh, prob.u0, prob.v0, precision, m_cap)
    return stream, ctx, mesh, traj


def test_footprint_matches_device_memory():
    """etp_traj_footprint counts what etp_state_init allocates (cudaMemGetInfo; each of the ~25
    allocations may round up to a 2 MiB page, less than any of the large buffers)."""
    import torch
    from paper_2405_05213_gb300 import etp
    prob = inputs.make_problem("rubber-neohooke-q2", n=24)
    stream = torch.cuda.Stream()
    ctx = etp.Context(0, stream=stream.cuda_stream)
    mesh = etp.Mesh.from_problem(ctx, prob)
    tb, mb = etp.etp_traj_footprint(mesh.h, etp.ETP_PREC_MIXED, 64)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    traj = etp.Trajectory(mesh, prob.u0, prob.v0, etp.ETP_PREC_MIXED, 64)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info(0)[0]
    assert tb <= used + 2**20 and used - tb <= 25 * 2 * 2**20, (used, tb)
    assert mb > 0
    traj.close(); mesh.close(); ctx.close()


def test_batch_steps_equal_direct_steps_and_failures_retire_alone():
    """The native batch gives the same state as stepping alone; a failing request retires with its status."""
    import time
    from paper_2405_05213_gb300 import etp
    mix = inputs.served_mix(3, dof_range=(2000, 20000), horizon=(5, 8))
    direct = []
    for arr, p, steps in mix:
        s, c, m, t = _objects(p, etp.ETP_PREC_MIXED)
        for _ in range(steps):
            t.step(p.dt, p.tol)
        direct.append(t.state())
        t.close(); m.close(); c.close()
    ctx = etp.Context(0)
    batch = etp.etp_batch_create(ctx.h, 1 << 40, 4)
    objs = [_objects(p, etp.ETP_PREC_MIXED) for arr, p, steps in mix]
    # a request that cannot converge: m_cap 2 at a tight tolerance
    arr, pf, _ = mix[0]
    fail_objs = _objects(pf, etp.ETP_PREC_MIXED, m_cap=2)
    for (arr, p, steps), o in zip(mix, objs):
        assert etp.etp_batch_admit(batch, o[3].h, steps, p.dt, p.tol)
    assert etp.etp_batch_admit(batch, fail_objs[3].h, 3, pf.dt, 1e-14)
    retired = {}
    t0 = time.time()
    while len(retired) < 4 and time.time() - t0 < 120:
        etp.etp_batch_tick(batch)
        for th, st in etp.etp_batch_retired(batch):
            retired[th] = st
    assert len(retired) == 4
    assert retired[fail_objs[3].h.value] == etp.ETP_ERR_NOT_CONVERGED
    for (arr, p, steps), o, (u, v) in zip(mix, objs, direct):
        assert retired[o[3].h.value] == etp.ETP_OK
        sd, st, rt, ms = etp.etp_batch_traj_info(batch, o[3].h)
        assert sd == steps and st == 0 and rt and ms.size == steps and (ms > 0).all()
        ub, vb = o[3].state()
        assert np.array_equal(ub, u) and np.array_equal(vb, v)
    reserved, n_active = etp.etp_batch_usage(batch)
    assert reserved == 0 and n_active == 0
    etp.etp_batch_destroy(batch)
    for o in objs + [fail_objs]:
        o[3].close(); o[2].close(); o[1].close()
    ctx.close()
