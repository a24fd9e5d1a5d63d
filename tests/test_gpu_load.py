"""Constant external load (Section 2.3, Eq. "A expression at P != 0") on the GPU, against the oracle.

Tolerances as in test_gpu_parity: FP64 1e-10 (linear) / 1e-8 (Neo-Hooke) relative L2 after the
horizon, MIXED 1e-5. Both the fused persistent Arnoldi step (short vectors) and the separate
gather + bulk-copy passes are exercised."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import inputs
from oracle import propagator

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def E():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp
    assert torch.cuda.is_available()
    return etp, etp.Context(0)


def _gpu(etp, ctx, p, precision, u0=None, v0=None, m_cap=64):
    mesh = etp.Mesh.from_problem(ctx, p)
    t = etp.Trajectory(mesh, p.u0 if u0 is None else u0, p.v0 if v0 is None else v0, precision, m_cap)
    t.set_load(p.load)
    return mesh, t


@pytest.mark.parametrize("fused", [True, False])
def test_linear_beam_with_load_fp64(E, fused, monkeypatch):
    etp, ctx = E
    if not fused:
        monkeypatch.setenv("ETP_NO_PERSISTENT", "1")  # read when a context is created
        ctx = etp.Context(0)
    p = inputs.with_face_load(inputs.beam_linear(), -0.5, comp=1)
    O = propagator.Propagator.from_problem(p)
    mesh, t = _gpu(etp, ctx, p, etp.ETP_PREC_FP64)
    for _ in range(40):
        O.step(p.dt, 1e-12)
        t.step(p.dt, 1e-12)
    u, v = t.state()
    assert rel(u, O.u_full()) <= 1e-10 and rel(v, O.v_full()) <= 1e-10
    eg, eo = t.energy(), O.energy()
    assert abs(eg[0] - eo[0]) <= 1e-10 * (eo[1] + abs(eo[2]))
    assert abs(eg[2] - eo[2]) <= 1e-10 * (eo[1] + abs(eo[2]))
    t.close(); mesh.close()


@pytest.mark.parametrize("precision,bar", [("FP64", 1e-8), ("MIXED", 1e-5)])
def test_neohooke_beam_with_load(E, precision, bar):
    etp, ctx = E
    base = inputs.beam_neohooke(nel=(10, 2, 2), dt=0.02, steps=20, jitter=False)
    p = inputs.with_face_load(base, -2.0, comp=1)
    O = propagator.Propagator.from_problem(p, m_cap=64)
    mesh, t = _gpu(etp, ctx, p, getattr(etp, "ETP_PREC_" + precision))
    for _ in range(20):
        O.step(p.dt, 1e-10)
        t.step(p.dt, 1e-10)
    u, v = t.state()
    assert rel(u, O.u_full()) <= bar and rel(v, O.v_full()) <= bar
    t.close(); mesh.close()


def test_static_equilibrium_under_load_stays_at_rest(E):
    """At R(u_s) = P with v = 0, A[u_s] [u_s; 0; 1] = 0: the GPU step leaves the state in place."""
    etp, ctx = E
    base = inputs.beam_neohooke(nel=(10, 2, 2), dt=0.02, steps=2, jitter=False)
    p = inputs.with_face_load(base, -2.0, comp=1)
    fe = propagator.Propagator.from_problem(p).fe
    u = np.zeros(fe.N)
    Pf = p.load[fe.free]
    for _ in range(30):  # Newton on the oracle side (the input, not an expected value of the GPU)
        r = fe.internal_force(p.material, p.params, u)[fe.free] - Pf
        if np.linalg.norm(r) <= 1e-12 * np.linalg.norm(Pf):
            break
        u[fe.free] -= spla.spsolve(fe.assemble_H(p.material, p.params, u, tangent=True).tocsc(), r)
    for prec, bar in ((etp.ETP_PREC_FP64, 1e-8), (etp.ETP_PREC_MIXED, 1e-4)):
        mesh, t = _gpu(etp, ctx, p, prec, u0=u, v0=np.zeros_like(u))
        for _ in range(2):
            t.step(p.dt, 1e-10)
        ug, vg = t.state()
        assert rel(ug, u) <= bar and np.linalg.norm(vg) <= bar * np.linalg.norm(u)
        t.close(); mesh.close()


def test_removing_the_load_restores_the_plain_state(E):
    etp, ctx = E
    p = inputs.with_face_load(inputs.beam_linear(), -0.5, comp=1)
    mesh = etp.Mesh.from_problem(ctx, p)
    a = etp.Trajectory(mesh, p.u0, p.v0, etp.ETP_PREC_FP64, 64)
    b = etp.Trajectory(mesh, p.u0, p.v0, etp.ETP_PREC_FP64, 64)
    a.set_load(p.load)
    a.set_load(None)
    for _ in range(5):
        a.step(p.dt, 1e-12)
        b.step(p.dt, 1e-12)
    ua, va = a.state()
    ub, vb = b.state()
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    a.close(); b.close(); mesh.close()
