"""Ragged batched step (etp_step_batch) on the GPU.

A mixed batch -- Q1 and Q2 meshes of different sizes, linear / Neo-Hooke / Mooney-Rivlin (with
element stiffness scales), FP64 and MIXED, its own dt and tol each, one under a constant load --
advances in lockstep with one element-pass launch per class and one persistent Arnoldi-step launch
per precision per Krylov iteration. Every kernel computes a trajectory's values as its single launch
does (per-element terms, per-tile partial sums summed in tile order, per-candidate exponentials), so
each trajectory must end BITWISE where etp_step_ex alone takes it, with the same Krylov sizes; the
single-trajectory path is itself checked against the FP64 oracle in test_gpu_parity / test_gpu_load.
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp
    assert torch.cuda.is_available()
    return etp


def _mix(etp):
    F64, MIX = etp.ETP_PREC_FP64, etp.ETP_PREC_MIXED
    lin = inputs.beam_linear()
    loaded = inputs.with_face_load(inputs.beam_linear(nel=(10, 2, 2)), total=0.5)
    nh = inputs.beam_neohooke(nel=(16, 2, 2), dt=0.02)
    nh_big = inputs.beam_neohooke(nel=(40, 4, 4), dt=0.02)
    rub = inputs.rubber_block(n=4)
    tis = inputs.tissue_slab(nel=(8, 4, 4))
    return [(lin, F64), (loaded, F64), (nh, F64), (nh, MIX), (nh_big, MIX), (rub, MIX), (tis, MIX),
            (tis, F64)]


def _make(etp, ctx, p, prec):
    mesh = etp.Mesh.from_problem(ctx, p)
    t = etp.Trajectory(mesh, p.u0, p.v0, prec, 64)
    if p.load is not None:
        t.set_load(p.load)
    return mesh, t


def test_batch_equals_alone_bitwise(E):
    etp = E
    mix = _mix(etp)
    steps = 4
    ctx_a = etp.Context(0)
    alone = []
    for p, prec in mix:
        mesh, t = _make(etp, ctx_a, p, prec)
        ms = []
        for _ in range(steps):
            _, info = t.step_ex(p.dt, p.tol)
            ms.append((info.m_pred, info.m_corr))
        alone.append((t.state(), ms, mesh, t))
    ctx_b = etp.Context(0)
    objs = [_make(etp, ctx_b, p, prec) for p, prec in mix]
    trajs = [t.h for _, t in objs]
    ms_b = [[] for _ in mix]
    for _ in range(steps):
        sts, infos = etp.etp_step_batch(trajs, [p.dt for p, _ in mix], [p.tol for p, _ in mix])
        assert all(s == etp.ETP_OK for s in sts)
        for k, inf in enumerate(infos):
            assert inf.converged == 1
            ms_b[k].append((inf.m_pred, inf.m_corr))
    for k, (p, prec) in enumerate(mix):
        ua, va = alone[k][0]
        ub, vb = objs[k][1].state()
        assert ms_b[k] == alone[k][1], (p.name, prec, ms_b[k], alone[k][1])
        assert np.array_equal(ua, ub) and np.array_equal(va, vb), (p.name, prec)
        assert np.linalg.norm(ub) > 0 or np.linalg.norm(vb) > 0
    e_a = [alone[k][3].energy() for k in range(len(mix))]
    e_b = [objs[k][1].energy() for k in range(len(mix))]
    assert e_a == e_b


def test_batch_of_one_and_repeated_batches(E):
    """A batch of one is etp_step_ex; stepping in batches of changing membership keeps each
    trajectory on its own path (the midpoint history is per trajectory)."""
    etp = E
    p = inputs.beam_neohooke(nel=(16, 2, 2), dt=0.02)
    q = inputs.rubber_block(n=4)
    ctx = etp.Context(0)
    _, ta = _make(etp, ctx, p, etp.ETP_PREC_MIXED)
    _, tb = _make(etp, ctx, p, etp.ETP_PREC_MIXED)
    _, tc = _make(etp, ctx, q, etp.ETP_PREC_MIXED)
    _, td = _make(etp, ctx, q, etp.ETP_PREC_MIXED)
    for step in range(5):
        ta.step_ex(p.dt, p.tol)
        tc.step_ex(q.dt, q.tol)
        group = [tb.h] + ([td.h] if step % 2 == 0 else [])
        dts = [p.dt] + ([q.dt] if step % 2 == 0 else [])
        tols = [p.tol] + ([q.tol] if step % 2 == 0 else [])
        etp.etp_step_batch(group, dts, tols)
        if step % 2 == 1:
            etp.etp_step_batch([td.h], [q.dt], [q.tol])
    for x, y in ((ta, tb), (tc, td)):
        ux, vx = x.state()
        uy, vy = y.state()
        assert np.array_equal(ux, uy) and np.array_equal(vx, vy)


def test_batch_argument_errors(E):
    etp = E
    p = inputs.beam_linear(nel=(6, 2, 2))
    c1, c2 = etp.Context(0), etp.Context(0)
    _, t1 = _make(etp, c1, p, etp.ETP_PREC_FP64)
    _, t2 = _make(etp, c2, p, etp.ETP_PREC_FP64)
    u0, v0 = t1.state()
    with pytest.raises(etp.EtpError):
        etp.etp_step_batch([t1.h, t2.h], [p.dt, p.dt], [p.tol, p.tol])
    with pytest.raises(etp.EtpError):
        etp.etp_step_batch([t1.h, t1.h], [p.dt, p.dt], [p.tol, p.tol])
    with pytest.raises(etp.EtpError):
        etp.etp_step_batch([t1.h], [-1.0], [p.tol])
    u1, v1 = t1.state()  # nothing was stepped
    assert np.array_equal(u0, u1) and np.array_equal(v0, v1)
    assert etp.etp_step_batch([], [], []) == ([], [])
