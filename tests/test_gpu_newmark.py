"""Newmark-beta on the GPU (etp_newmark_step, Section 6's comparison integrator) against the
oracle's Newmark-beta (sparse direct solves), FP64. Linear: relative L2 <= 1e-10 in u and v after the
horizon (CG to a relative residual of 1e-13 per step); average acceleration conserves the energy of
the undamped linear system; the state does not depend on the trajectory's Krylov precision. SVK,
Neo-Hooke, Mooney-Rivlin and Yeoh ("fully implicit", Newton with the consistent tangent on both
sides, the GPU's CG-solved): relative L2 <= 1e-9 after the horizon."""
import numpy as np
import pytest

import inputs
from oracle.newmark import Newmark

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def etp():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp
    assert torch.cuda.is_available()
    return etp


def _traj(etp, ctx, p, prec):
    mesh = etp.Mesh.from_problem(ctx, p)
    return mesh, etp.Trajectory(mesh, p.u0, p.v0, prec, 16)


@pytest.mark.parametrize("nel,dt,steps", [((20, 2, 2), 0.05, 40), ((12, 3, 3), 0.01, 25)])
def test_newmark_matches_oracle(etp, nel, dt, steps):
    p = inputs.beam_linear(nel=nel)
    ctx = etp.Context(0)
    mesh, t = _traj(etp, ctx, p, etp.ETP_PREC_FP64)
    N = Newmark.from_problem(p)
    E0 = t.energy()[0]
    iters = []
    for _ in range(steps):
        iters.append(etp.etp_newmark_step(t.h, dt, 1e-13))
        N.step(dt)
    u, v = t.state()
    assert rel(u, N.fe.to_full(N.u)) < 1e-10
    assert rel(v, N.fe.to_full(N.v)) < 1e-10
    assert abs(t.energy()[0] - E0) / E0 < 1e-9
    assert max(iters) > 0


@pytest.mark.parametrize("kind", ["linear", "svk"])
def test_newmark_graph_replay_equals_direct_launches(etp, kind, monkeypatch):
    """On a created stream the CG blocks replay a captured CUDA graph: same bits as launching them."""
    import torch
    p = inputs.beam_linear(nel=(16, 2, 2)) if kind == "linear" else _svk_beam((12, 2, 2), 0.02)
    st = torch.cuda.Stream()
    ctx = etp.Context(0, stream=st.cuda_stream)
    _, a = _traj(etp, ctx, p, etp.ETP_PREC_FP64)
    for dt in (0.02, 0.02, 0.01, 0.01):  # a change of dt recaptures
        etp.etp_newmark_step(a.h, dt, 1e-12)
    monkeypatch.setenv("ETP_NO_GRAPHS", "1")  # read when a context is created
    ctx_direct = etp.Context(0, stream=st.cuda_stream)
    _, b = _traj(etp, ctx_direct, p, etp.ETP_PREC_FP64)
    for dt in (0.02, 0.02, 0.01, 0.01):
        etp.etp_newmark_step(b.h, dt, 1e-12)
    ua, va = a.state()
    ub, vb = b.state()
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    assert np.linalg.norm(ua) > 0


def test_newmark_state_independent_of_krylov_precision_and_mixes_with_propagator(etp):
    p = inputs.beam_linear()
    ctx = etp.Context(0)
    _, a = _traj(etp, ctx, p, etp.ETP_PREC_FP64)
    _, b = _traj(etp, ctx, p, etp.ETP_PREC_MIXED)
    for _ in range(10):
        etp.etp_newmark_step(a.h, 0.02, 1e-12)
        etp.etp_newmark_step(b.h, 0.02, 1e-12)
    ua, va = a.state()
    ub, vb = b.state()
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    # a propagator step in between: the acceleration is recomputed from the new state, so the
    # result matches the oracle's Newmark restarted from that state
    a.step(0.02, 1e-12)
    u1, v1 = a.state()
    q = inputs.beam_linear()
    q.u0, q.v0 = u1, v1
    N = Newmark.from_problem(q)
    for _ in range(5):
        etp.etp_newmark_step(a.h, 0.02, 1e-13)
        N.step(0.02)
    u2, v2 = a.state()
    assert rel(u2, N.fe.to_full(N.u)) < 1e-10 and rel(v2, N.fe.to_full(N.v)) < 1e-10


def _svk_beam(nel, dt):
    import dataclasses
    p = inputs.beam_neohooke(nel=nel, dt=dt, amp_scale=2.0)
    return dataclasses.replace(p, name="beam-svk-q1", material=inputs.MAT_SVK, params=(805.0, 345.0))


@pytest.mark.parametrize("prec_name", ["ETP_PREC_FP64", "ETP_PREC_MIXED"])
def test_newmark_svk_matches_oracle(etp, prec_name):
    p = _svk_beam((12, 2, 2), 0.02)
    ctx = etp.Context(0)
    mesh, t = _traj(etp, ctx, p, getattr(etp, prec_name))
    N = Newmark.from_problem(p)
    for _ in range(15):
        etp.etp_newmark_step(t.h, 0.02, 1e-12)
        N.step(0.02)
    u, v = t.state()
    assert np.linalg.norm(u) > 0
    assert rel(u, N.fe.to_full(N.u)) < 1e-9
    assert rel(v, N.fe.to_full(N.v)) < 1e-9


@pytest.mark.parametrize("kind,params", [(inputs.MAT_NEOHOOKE, (345.0, 805.0)),
                                         (inputs.MAT_MOONEY_RIVLIN, (0.5, 0.05, 1.1e3)),
                                         (inputs.MAT_YEOH, (100.0, -1.0, 0.01, 0.001))])
def test_newmark_hyperelastic_matches_oracle(etp, kind, params):
    """Neo-Hooke, Mooney-Rivlin and Yeoh (the paper's tissue and rubber material, Tables 3-4):
    the GPU's Newton iterations use the exact tangent dP/dF (dual-number differentiation of
    P(F)), the oracle's a central-difference one; both converge to the same implicit step."""
    p = inputs.tissue_slab(nel=(8, 4, 4), steps=0)
    p.material, p.params = kind, params
    p.v0 = 5.0 * p.v0
    dt = inputs.cfl_dt(p.mesh, kind, params, 1.0, 2.0)
    ctx = etp.Context(0)
    mesh, t = _traj(etp, ctx, p, etp.ETP_PREC_FP64)
    N = Newmark.from_problem(p)
    for _ in range(10):
        etp.etp_newmark_step(t.h, dt, 1e-12)
        N.step(dt)
    u, v = t.state()
    assert np.linalg.norm(u) > 0
    assert rel(u, N.fe.to_full(N.u)) < 1e-9 and rel(v, N.fe.to_full(N.v)) < 1e-9, \
        (rel(u, N.fe.to_full(N.u)), rel(v, N.fe.to_full(N.v)))


@pytest.mark.parametrize("kind,params", [(inputs.MAT_SVK, (805.0, 345.0)),
                                         (inputs.MAT_NEOHOOKE, (345.0, 805.0)),
                                         (inputs.MAT_MOONEY_RIVLIN, (0.5, 0.05, 1.1e3)),
                                         (inputs.MAT_YEOH, (100.0, -1.0, 0.01, 0.001))])
@pytest.mark.parametrize("perturb", [False, True])
def test_consistent_tangent_matches_oracle(etp, kind, params, perturb):
    """The GPU tangent operator (closed form for SVK, dual-number dP/dF otherwise) against the
    oracle's assembled dR/du (central differences of P, itself pinned to finite differences of
    the internal force) at a finitely strained state."""
    from oracle import fem
    mesh = inputs.box_mesh(1, 5, 3, 3, 2.0, 1.0, 1.0)
    if perturb:
        mesh = inputs.perturb_interior(mesh, 5)
    fixed = inputs.fixed_dofs_on_plane(mesh, 0, 0.0)
    rng = np.random.default_rng(17)
    scale = np.exp(0.1 * rng.standard_normal(mesh.n_elems)).astype(np.float32)
    d = fem.Discretisation(1, mesh.coords, mesh.conn, fixed, 1.2, scale)
    u = d.to_full(0.03 * rng.standard_normal(d.Nf))
    x = d.to_full(rng.standard_normal(d.Nf))
    KT = d.scaled(d.assemble_H(kind, params, u, tangent=True))
    ref = KT @ x[d.free]
    ctx = etp.Context(0)
    m = etp.Mesh(ctx, 1, mesh.coords, mesh.conn, fixed)
    m.set_material(kind, params, 1.2, scale)
    y = etp.etp_apply_tangent(m.h, x, u)
    assert np.all(y[d.fixed] == 0.0)
    assert rel(y[d.free], ref) < 1e-7, rel(y[d.free], ref)


def test_newmark_rejects_a_load_and_bad_arguments(etp):
    ctx = etp.Context(0)
    p = inputs.with_face_load(inputs.beam_neohooke(nel=(8, 2, 2), dt=0.02), -1.0)
    _, t = _traj(etp, ctx, p, etp.ETP_PREC_FP64)
    t.set_load(p.load)
    with pytest.raises(etp.EtpError):
        etp.etp_newmark_step(t.h, 0.02, 1e-12)
    q = inputs.beam_linear(nel=(6, 2, 2))
    _, s = _traj(etp, ctx, q, etp.ETP_PREC_FP64)
    with pytest.raises(etp.EtpError):
        etp.etp_newmark_step(s.h, -1.0, 1e-12)
    with pytest.raises(etp.EtpError):
        etp.etp_newmark_step(s.h, 0.02, 0.0)
