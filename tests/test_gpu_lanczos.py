"""Energy-inner-product Lanczos (ETP_KRYLOV_LANCZOS_ENERGY) through the C ABI.

For a linear material H_bar is symmetric positive definite and A is skew-adjoint in the energy
inner product (Section 4.3, Section 5.2 Eq. "energyExpr"), so the Krylov process reduces to a
three-term recurrence. Checks: the propagated state equals the oracle's Arnoldi result (same
problem, tight tolerances) and the dense exp(dt A) w on a tiny mesh; energy is conserved; the
process moves far fewer vector bytes than the Gram-Schmidt passes; misuse is rejected.
"""
import numpy as np
import pytest
import scipy.linalg

import inputs
from oracle import materials, propagator

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


def _traj(etp, ctx, p, prec, m_cap=128, u0=None, v0=None):
    mesh = etp.Mesh.from_problem(ctx, p)
    t = etp.Trajectory(mesh, p.u0 if u0 is None else u0, p.v0 if v0 is None else v0, prec, m_cap)
    t.set_krylov(etp.ETP_KRYLOV_LANCZOS_ENERGY)
    return mesh, t


def test_matches_dense_exponential_on_a_tiny_mesh(E):
    """exp(dt A) w by scipy's dense expm on a 2x1x1 beam (90 free DOFs), several dt."""
    etp, ctx = E
    mesh = inputs.box_mesh(1, 4, 2, 2, 2.0, 1.0, 1.0)
    fixed = inputs.fixed_dofs_on_plane(mesh, 0, 0.0)
    rng = np.random.default_rng(3)
    u0 = 1e-2 * rng.standard_normal(3 * mesh.n_nodes)
    v0 = rng.standard_normal(3 * mesh.n_nodes)
    u0[fixed] = 0.0
    v0[fixed] = 0.0
    P = propagator.Propagator(1, mesh.coords, mesh.conn, fixed, materials.LINEAR, (1e3, 0.3), 1.0, u0, v0)
    Hb = P.Hbar(None).toarray()
    Nf = P.Nf
    A = np.block([[np.zeros((Nf, Nf)), np.eye(Nf)], [-Hb, np.zeros((Nf, Nf))]])
    m = etp.Mesh(ctx, 1, mesh.coords, mesh.conn, fixed)
    m.set_material(materials.LINEAR, (1e3, 0.3), 1.0)
    for dt in (0.002, 0.02, 0.1):
        w = scipy.linalg.expm(dt * A) @ P.w
        u_ref, v_ref = P.u_full(w), P.v_full(w)
        t = etp.Trajectory(m, u0, v0, etp.ETP_PREC_FP64, 180)
        t.set_krylov(etp.ETP_KRYLOV_LANCZOS_ENERGY)
        st, info = t.step_ex(dt, 1e-13)
        u, v = t.state()
        assert rel(u, u_ref) < 1e-9 and rel(v, v_ref) < 1e-9, (dt, rel(u, u_ref), rel(v, v_ref), info.m_corr)
        t.close()


@pytest.mark.parametrize("prec_name,bar", [("FP64", (1e-9, 1e-9)), ("MIXED", (1e-5, 2e-4))])
def test_linear_beam_200_steps_against_oracle_arnoldi(E, prec_name, bar):
    """Config 1 horizon: the oracle's Arnoldi (tol 1e-12) against the GPU Lanczos (tol 1e-12).
    MIXED: u within 1e-5, v within 2e-4 (the FP32 operator's cancellation on smooth fields, as
    for the Arnoldi MIXED form)."""
    etp, ctx = E
    p = inputs.beam_linear()
    O = propagator.Propagator.from_problem(p)
    for _ in range(p.steps):
        O.step(p.dt, 1e-12)
    _, t = _traj(etp, ctx, p, getattr(etp, f"ETP_PREC_{prec_name}"))
    E0 = t.energy()[0]
    for _ in range(p.steps):
        st, info = t.step_ex(p.dt, 1e-12)
        assert info.converged
    u, v = t.state()
    assert rel(u, O.u_full()) < bar[0] and rel(v, O.v_full()) < bar[1], (rel(u, O.u_full()), rel(v, O.v_full()))
    assert abs(t.energy()[0] - E0) / E0 < (1e-9 if prec_name == "FP64" else 1e-5)


def test_config_tolerance_and_sizes(E):
    """At the config's tolerance (1e-10) the Lanczos sizes are those of Arnoldi within a few
    (the estimate is measured in the energy norm instead of the Euclidean one) and the states
    agree to the tolerance."""
    etp, ctx = E
    p = inputs.beam_linear()
    steps = 50
    O = propagator.run(p, steps=steps)
    _, t = _traj(etp, ctx, p, etp.ETP_PREC_FP64)
    ms = []
    for _ in range(steps):
        st, info = t.step_ex(p.dt, p.tol)
        ms.append(info.m_corr)
        assert info.converged and info.eps_corr <= p.tol * info.beta
    assert all(abs(a - b) <= 3 for a, b in zip(ms, O.log.m)), (ms, O.log.m)
    u, v = t.state()
    assert rel(u, O.u_full()) < 1e-8 and rel(v, O.v_full()) < 1e-8


def test_vector_bytes_far_below_gram_schmidt(E):
    """Same linear slab (2.2M rows, Gram-Schmidt bulk passes) with Arnoldi and with Lanczos: the
    Lanczos vector passes move a small fraction of the Gram-Schmidt bytes, and both states agree
    within the tolerance."""
    etp, ctx = E
    base = inputs.tissue_slab(nel=(128, 64, 48), steps=0)
    lam, mu = 1.1e3 - 2.0 * 1.1 / 3.0, 1.1
    E_ = mu * (3 * lam + 2 * mu) / (lam + mu)
    nu = lam / (2 * (lam + mu))
    base.material, base.params = materials.LINEAR, (E_, nu)
    mesh = etp.Mesh.from_problem(ctx, base)
    out = {}
    for name, method in (("arnoldi", etp.ETP_KRYLOV_ARNOLDI), ("lanczos", etp.ETP_KRYLOV_LANCZOS_ENERGY)):
        t = etp.Trajectory(mesh, base.u0, base.v0, etp.ETP_PREC_MIXED, 64)
        t.set_krylov(method)
        t.step(base.dt, base.tol)
        etp.etp_profile_reset(ctx.h)
        etp.etp_profile_enable(ctx.h, True)
        for _ in range(2):
            t.step(base.dt, base.tol)
        etp.etp_profile_enable(ctx.h, False)
        prof = etp.etp_profile_read(ctx.h)
        out[name] = (t.state(), prof)
        t.close()
    gs = sum(out["arnoldi"][1][k]["bytes"] for k in ("cgs_dot", "cgs_update_dot", "cgs_update_norm"))
    lz = out["lanczos"][1]["lanczos"]["bytes"]
    assert out["lanczos"][1]["cgs_dot"]["launches"] == 0 and lz > 0
    assert lz < 0.25 * gs, (lz, gs)
    (ua, va), (ub, vb) = out["arnoldi"][0], out["lanczos"][0]
    assert rel(ub, ua) < 1e-4 and rel(vb, va) < 1e-4


def test_rejected_where_the_operator_is_not_skew_adjoint(E):
    etp, ctx = E
    p = inputs.beam_neohooke(nel=(8, 2, 2), dt=0.05)
    mesh = etp.Mesh.from_problem(ctx, p)
    t = etp.Trajectory(mesh, p.u0, p.v0, etp.ETP_PREC_FP64, 32)
    with pytest.raises(etp.EtpError):
        t.set_krylov(etp.ETP_KRYLOV_LANCZOS_ENERGY)
    with pytest.raises(etp.EtpError):
        t.set_krylov(7)
    pl = inputs.with_face_load(inputs.beam_linear(), -0.5, comp=1)
    _, tl = _traj(etp, ctx, pl, etp.ETP_PREC_FP64)
    tl.set_load(pl.load)
    st, _ = tl.step_ex(pl.dt, pl.tol, check=False)
    assert st == etp.ETP_ERR_INVALID and tl.steps == 0
