"""Failure detection through the C ABI, with every failure made on the host side.

* A bounded wait that runs out: the test hook etp_debug_spin_limit lowers the
  poll limit of the persistent Arnoldi step's grid barrier, so the waiting
  blocks give up (no kernel is left waiting: each records the timeout and
  ends). The step must return ETP_ERR_TIMEOUT without committing anything, and
  the next step (built-in limit again) must equal that of a trajectory that
  never failed, bit for bit.
* A non-finite input (NaN in the initial velocity) -> ETP_ERR_NONFINITE.
* A frozen state with an inverted element (det F <= 0 built on the host)
  -> ETP_ERR_INVERTED_ELEMENT.
In every case the state, the step count and the predictor history stay as
they were.
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def etp():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp as mod
    assert torch.cuda.is_available()
    return mod


def _traj(etp, ctx, p, prec, u0=None, v0=None):
    mesh = etp.Mesh.from_problem(ctx, p)
    return mesh, etp.Trajectory(mesh, p.u0 if u0 is None else u0, p.v0 if v0 is None else v0, prec, p.m_cap)


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED"])
def test_barrier_timeout_is_reported_and_not_committed(etp, prec_name):
    prec = getattr(etp, f"ETP_PREC_{prec_name}")
    ctx = etp.Context(0)
    # the config-2 beam: ~40k-row vectors, so the persistent step runs on many blocks
    p = inputs.beam_neohooke(dt=0.02)
    _, a = _traj(etp, ctx, p, prec)
    _, b = _traj(etp, ctx, p, prec)
    for _ in range(2):
        a.step(p.dt, p.tol)
        b.step(p.dt, p.tol)
    u0, v0 = a.state()
    etp.etp_debug_spin_limit(ctx.h, 1)
    try:
        st, _ = a.step_ex(p.dt, p.tol, check=False)
    finally:
        etp.etp_debug_spin_limit(ctx.h, 0)
    assert st == etp.ETP_ERR_TIMEOUT
    assert "timed out" in etp.lib().etp_last_error().decode()
    u1, v1 = a.state()
    assert np.array_equal(u0, u1) and np.array_equal(v0, v1)
    assert a.steps == 2
    # the barrier words were reset: the trajectory goes on as if nothing happened
    for _ in range(2):
        a.step(p.dt, p.tol)
        b.step(p.dt, p.tol)
    ua, va = a.state()
    ub, vb = b.state()
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
    assert a.steps == 4


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED"])
def test_nonfinite_initial_velocity(etp, prec_name):
    prec = getattr(etp, f"ETP_PREC_{prec_name}")
    ctx = etp.Context(0)
    p = inputs.beam_neohooke(nel=(16, 2, 2), dt=0.05)
    v0 = p.v0.copy()
    free = np.setdiff1d(np.arange(p.n_dofs), p.fixed_dofs)
    v0[free[len(free) // 2]] = np.nan
    _, t = _traj(etp, ctx, p, prec, v0=v0)
    st, _ = t.step_ex(p.dt, p.tol, check=False)
    assert st == etp.ETP_ERR_NONFINITE
    assert t.steps == 0
    u, v = t.state()
    assert np.array_equal(u, p.u0) and np.isnan(v[free[len(free) // 2]])


@pytest.mark.parametrize("prec_name", ["FP64", "MIXED"])
def test_inverted_element_in_frozen_state(etp, prec_name):
    """u0 that folds one element inside out: det F* <= 0 at its Gauss points when the predictor
    freezes u_0 (Section 4.2), so the step must stop with ETP_ERR_INVERTED_ELEMENT."""
    prec = getattr(etp, f"ETP_PREC_{prec_name}")
    ctx = etp.Context(0)
    p = inputs.beam_neohooke(nel=(16, 2, 2), dt=0.05)
    u0 = np.zeros(p.n_dofs)
    # push the far-x face nodes of element e (away from the clamp) past its near-x face
    e = p.mesh.n_elems // 2
    conn = p.mesh.conn[e]
    hx = p.mesh.lengths[0] / p.mesh.nel[0]
    for a in (1, 3, 5, 7):  # local nodes with a = 1 (x = +1 side), lexicographic order
        u0[3 * conn[a]] = -2.5 * hx
    _, t = _traj(etp, ctx, p, prec, u0=u0)
    st, _ = t.step_ex(p.dt, p.tol, check=False)
    assert st == etp.ETP_ERR_INVERTED_ELEMENT
    assert t.steps == 0
    u, v = t.state()
    np.testing.assert_allclose(u, u0, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(v, p.v0, rtol=1e-14, atol=1e-16)
