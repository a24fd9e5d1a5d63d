"""Autotuner (etp_autotune) on the GPU: it stores launch shapes, they are used, and the results stay
within the parity tolerances of test_gpu_parity (element results do not depend on the grid; the
Gram-Schmidt partial sums are grouped differently, a rounding-level change)."""
import numpy as np
import pytest

import inputs

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


@pytest.mark.parametrize("prec_name,tol", [("ETP_PREC_FP64", 1e-12), ("ETP_PREC_MIXED", 1e-5)])
def test_autotuned_shapes_keep_results(etp, prec_name, tol, monkeypatch):
    # separate Gram-Schmidt passes (as for vectors of more than 2^20 rows) on a mesh size no other
    # test uses, so the process-wide tuned shapes touch nothing else
    monkeypatch.setenv("ETP_NO_PERSISTENT", "1")
    prec = getattr(etp, prec_name)
    p = inputs.beam_neohooke(nel=(22, 3, 3), dt=0.02)
    ctx = etp.Context(0)
    mesh = etp.Mesh.from_problem(ctx, p)
    ref = etp.Trajectory(mesh, p.u0, p.v0, prec, 64)
    for _ in range(3):
        ref.step(p.dt, p.tol)
    u_ref, v_ref = ref.state()
    t = etp.Trajectory(mesh, p.u0, p.v0, prec, 64)
    s0 = t.state()
    n = etp.etp_autotune(t.h, 2)
    assert n >= 4  # element grids for 1 and 2 frozen states, and Gram-Schmidt shapes
    s1 = t.state()
    assert np.array_equal(s0[0], s1[0]) and np.array_equal(s0[1], s1[1])  # the state is untouched
    for _ in range(3):
        t.step(p.dt, p.tol)
    u, v = t.state()
    assert rel(u, u_ref) < tol and rel(v, v_ref) < tol
    # a second trajectory of the same shape uses the stored shapes: same bits as the tuned one
    t2 = etp.Trajectory(mesh, p.u0, p.v0, prec, 64)
    for _ in range(3):
        t2.step(p.dt, p.tol)
    u2, v2 = t2.state()
    assert np.array_equal(u, u2) and np.array_equal(v, v2)


def test_autotune_argument_errors(etp):
    p = inputs.beam_linear(nel=(6, 2, 2))
    ctx = etp.Context(0)
    mesh = etp.Mesh.from_problem(ctx, p)
    t = etp.Trajectory(mesh, p.u0, p.v0, etp.ETP_PREC_FP64, 16)
    with pytest.raises(etp.EtpError):
        etp.etp_autotune(t.h, 0)
