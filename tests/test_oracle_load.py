"""Pins for the oracle's constant external load (Section 2.3, Eq. "A expression at P != 0"): the
augmented state [u_bar; v_bar; 1] with the P_bar column, checked against what the mechanics fixes."""
import numpy as np
import scipy.sparse.linalg as spla

import inputs
from oracle import materials, propagator


def _loaded_linear(total=-0.5):
    return inputs.with_face_load(inputs.beam_linear(), total, comp=1)


def test_linear_load_matches_static_plus_free_vibration():
    """Linear, constant P: u(t) = u_s + (free vibration of u0 - u_s, v0) with K u_s = P
    (dense eigen-decomposition and solve: library routines, not the Krylov path)."""
    p = _loaded_linear()
    P = propagator.Propagator.from_problem(p)
    Nf = P.Nf
    H = P.Hbar(None).toarray()
    us = np.linalg.solve(H, P.pbar)  # static state in scaled form: H_bar u_s = P_bar
    lam, Q = np.linalg.eigh(H)
    om = np.sqrt(lam)
    a = Q.T @ (P.w[:Nf] - us)
    b = Q.T @ P.w[Nf:2 * Nf]
    steps, dt = 40, p.dt
    for _ in range(steps):
        P.step(dt, 1e-12)
    t = steps * dt
    ub = us + Q @ (np.cos(om * t) * a + np.sin(om * t) / om * b)
    vb = Q @ (-om * np.sin(om * t) * a + np.cos(om * t) * b)
    assert np.linalg.norm(P.w[:Nf] - ub) <= 1e-10 * np.linalg.norm(ub)
    assert np.linalg.norm(P.w[Nf:2 * Nf] - vb) <= 1e-10 * np.linalg.norm(vb)
    assert abs(P.w[-1] - 1.0) <= 1e-12  # the augmented entry stays 1


def test_linear_load_conserves_energy_with_load_potential():
    """E = v'v/2 + u'Hu/2 - P'u is conserved by exp(dt A); Krylov adds at most ~tol per step."""
    p = _loaded_linear()
    P = propagator.Propagator.from_problem(p)
    Nf = P.Nf
    Hb = P.Hbar(None)

    def mechanical(w):  # kinetic + strain energy, without the load potential
        return 0.5 * w[Nf:2 * Nf] @ w[Nf:2 * Nf] + 0.5 * w[:Nf] @ (Hb @ w[:Nf])
    E0, K0, U0 = P.energy()
    M0 = mechanical(P.w)
    scale = K0 + abs(U0)
    for _ in range(50):
        P.step(p.dt, p.tol)
    assert abs(P.energy()[0] - E0) <= 10 * p.tol * 50 * scale
    # the load does work: the mechanical energy alone changes
    assert abs(mechanical(P.w) - M0) > 1e-3 * scale


def test_zero_load_gives_the_unloaded_motion():
    p = inputs.beam_linear()
    p0 = inputs.with_face_load(p, 0.0)
    A = propagator.Propagator.from_problem(p)
    B = propagator.Propagator.from_problem(p0)
    for _ in range(10):
        A.step(p.dt, 1e-13)
        B.step(p.dt, 1e-13)
    Nf = A.Nf
    assert np.linalg.norm(A.w - B.w[:2 * Nf]) <= 1e-11 * np.linalg.norm(A.w)


def test_nonlinear_static_equilibrium_stays_at_rest():
    """Neo-Hooke at the static state R(u_s) = P, v = 0: since H(u_s) u_s = R(u_s) (the split's
    defining property), A[u_s] [u_s; 0; 1] = 0 and the step must leave the state unchanged."""
    base = inputs.beam_neohooke(nel=(10, 2, 2), dt=0.02, steps=2, jitter=False)
    p = inputs.with_face_load(base, -2.0, comp=1)
    P0 = propagator.Propagator.from_problem(p)
    fe = P0.fe
    u = np.zeros(fe.N)
    Pf = p.load[fe.free]
    for _ in range(30):  # Newton on R(u) = P with the consistent tangent
        r = fe.internal_force(p.material, p.params, u)[fe.free] - Pf
        if np.linalg.norm(r) <= 1e-12 * np.linalg.norm(Pf):
            break
        Kt = fe.assemble_H(p.material, p.params, u, tangent=True)
        u[fe.free] -= spla.spsolve(Kt.tocsc(), r)
    r = fe.internal_force(p.material, p.params, u)[fe.free] - Pf
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(Pf)
    assert np.abs(u).max() > 1e-3  # a real deflection
    P = propagator.Propagator(p.mesh.order, p.mesh.coords, p.mesh.conn, p.fixed_dofs, p.material, p.params,
                              p.rho, u, np.zeros_like(u), load=p.load, m_cap=64)
    w0 = P.w.copy()
    for _ in range(2):
        P.step(p.dt, 1e-12)
    Nf = P.Nf
    assert np.linalg.norm(P.w[:Nf] - w0[:Nf]) <= 1e-8 * np.linalg.norm(w0[:Nf])
    assert np.linalg.norm(P.w[Nf:2 * Nf]) <= 1e-8 * np.linalg.norm(w0[:Nf])
