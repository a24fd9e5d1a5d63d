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


def test_admission_respects_memory_budget():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import serve
    mix = inputs.served_mix(4, dof_range=(2000, 8000), horizon=(2, 3))
    reqs = [serve.Request(k, 0.0, p, steps) for k, (arr, p, steps) in enumerate(mix)]
    need = max(serve.device_bytes_needed(r.problem, r.precision, r.m_cap) for r in reqs)
    srv = serve.Server(slots=4, memory_budget=int(1.5 * need), keep_state=False)
    peak = {"v": 0}
    orig = srv._run_one

    def spy(req, need_, t0):
        with srv._lock:
            peak["v"] = max(peak["v"], srv._reserved)
        orig(req, need_, t0)
    srv._run_one = spy
    res = srv.run(reqs, realtime=False)
    assert len(res) == 4 and all(r.status == "ok" for r in res.values())
    assert peak["v"] <= 1.5 * need
    big = serve.Server(slots=2, memory_budget=1024)
    big.run(reqs[:1], realtime=False)
    assert big.rejected == [0]
