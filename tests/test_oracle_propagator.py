"""Pins for the oracle's time step (no GPU): closed forms and the paper's stated properties."""
import numpy as np
import pytest
import scipy.linalg

import inputs
from oracle import materials, propagator
from oracle.newmark import Newmark


def _modal(P, w0, t):
    """Exact linear solution, Eq. "e^OmegaBt": cos/sin of sqrt(H_bar) on the modal basis."""
    Nf = P.Nf
    lam, Q = np.linalg.eigh(P.Hbar(None).toarray())
    om = np.sqrt(lam)
    a = Q.T @ w0[:Nf]
    b = Q.T @ w0[Nf:]
    ub = Q @ (np.cos(om * t) * a + np.sin(om * t) / om * b)
    vb = Q @ (-om * np.sin(om * t) * a + np.cos(om * t) * b)
    return ub, vb


def test_linear_beam_matches_modal_solution():
    p = inputs.beam_linear()
    P = propagator.Propagator.from_problem(p)
    w0 = P.w.copy()
    E0 = P.energy()[0]
    for _ in range(p.steps):
        P.step(p.dt, 1e-12)
    ub, vb = _modal(P, w0, p.steps * p.dt)
    Nf = P.Nf
    assert np.linalg.norm(P.w[:Nf] - ub) <= 1e-10 * np.linalg.norm(ub)
    assert np.linalg.norm(P.w[Nf:] - vb) <= 1e-10 * np.linalg.norm(vb)
    assert abs(P.energy()[0] - E0) <= 1e-10 * E0


def test_linear_energy_conservation_at_config_tolerance():
    """Section 5.2: exp(dt A) conserves E exactly; Krylov adds at most ~tol per step."""
    p = inputs.beam_linear()
    P = propagator.Propagator.from_problem(p)
    E0 = P.energy()[0]
    for _ in range(p.steps):
        P.step(p.dt, p.tol)
    assert abs(P.energy()[0] - E0) / E0 <= 10 * p.tol * p.steps
    assert all(P.log.converged)


def test_linear_step_has_no_time_error():
    """Linear problems: the Magnus series is exact, so one long step equals many short ones."""
    p = inputs.beam_linear()
    A = propagator.Propagator.from_problem(p)
    B = propagator.Propagator.from_problem(p)
    A.step(0.5, 1e-13)
    for _ in range(10):
        B.step(0.05, 1e-13)
    assert np.linalg.norm(A.w - B.w) <= 1e-10 * np.linalg.norm(B.w)


def test_symplectic_one_step_map():
    """Eq. "symplectic condition": Phi^T J Phi = J for the linear one-step map."""
    mesh = inputs.box_mesh(1, 2, 1, 1, 2.0, 1.0, 1.0)
    fixed = inputs.fixed_dofs_on_plane(mesh, 0, 0.0)
    z = np.zeros(3 * mesh.n_nodes)
    P = propagator.Propagator(1, mesh.coords, mesh.conn, fixed, materials.LINEAR, (1e3, 0.3), 1.0, z, z,
                              m_cap=200)
    n = 2 * P.Nf
    Phi = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        Phi[:, k] = P.expv(P.Hbar(None), 0.05, e, 1e-15).w
    Nf = P.Nf
    J = np.block([[np.zeros((Nf, Nf)), np.eye(Nf)], [-np.eye(Nf), np.zeros((Nf, Nf))]])
    assert np.abs(Phi.T @ J @ Phi - J).max() < 1e-12
    # and Phi is the exponential of dt A (closed form, Eq. "Jacobian")
    Hb = P.Hbar(None).toarray()
    A = np.block([[np.zeros((Nf, Nf)), np.eye(Nf)], [-Hb, np.zeros((Nf, Nf))]])
    np.testing.assert_allclose(Phi, scipy.linalg.expm(0.05 * A), atol=1e-12)


def _small_nh_beam(dt):
    return inputs.beam_neohooke(nel=(16, 2, 2), dt=dt, steps=0)


def test_nonlinear_second_order_in_dt():
    """Section 3.3 Eq. "timeDiscError", Section 5.1: global error at least O(dt^2).

    A smooth initial velocity (first bending mode, no nodal jitter) keeps the
    solution in the asymptotic regime; the abstract reports "quadratic and
    superquadratic" convergence, so the slope has a lower bound only.
    """
    T = 4.0

    def run(dt):
        P = propagator.Propagator.from_problem(
            inputs.beam_neohooke(nel=(16, 2, 2), dt=dt, steps=0, jitter=False))
        for _ in range(int(round(T / dt))):
            P.step(dt, 1e-13)
        return P
    ref = run(0.00625)
    errs = []
    for dt in [0.1, 0.05, 0.025]:
        P = run(dt)
        errs.append([np.linalg.norm(P.u_full() - ref.u_full()) / np.linalg.norm(ref.u_full()),
                     np.linalg.norm(P.v_full() - ref.v_full()) / np.linalg.norm(ref.v_full())])
    errs = np.array(errs)
    slopes = np.log(errs[:-1] / errs[1:]) / np.log(2.0)
    assert np.all(slopes > 1.8), (errs, slopes)
    assert np.all(slopes < 4.5), (errs, slopes)


def test_nonlinear_energy_drift_small():
    p = _small_nh_beam(0.05)
    P = propagator.Propagator.from_problem(p)
    E0 = P.energy()[0]
    for _ in range(40):
        P.step(0.05, 1e-10)
    assert abs(P.energy()[0] - E0) / E0 < 1e-4


def _rk4_reference(prob, dt_rk, n_steps, keep=None):
    """Split-independent reference: classical RK4 on M u'' = -R(u) (Section 2.2, Eq. "discrete
    dynamic equilibrium"), with R the internal force of the full constitutive law (no H-split)
    and the GLL mass. Returns {step: (u_free, v_free)} for the steps in `keep` (default: last)."""
    P = propagator.Propagator.from_problem(prob)
    fe = P.fe
    keep = {n_steps} if keep is None else set(keep)

    def acc(u):
        return -fe.internal_force(prob.material, prob.params, fe.to_full(u))[fe.free] / fe.mf

    u = np.asarray(prob.u0, dtype=np.float64)[fe.free].copy()
    v = np.asarray(prob.v0, dtype=np.float64)[fe.free].copy()
    out = {0: (u.copy(), v.copy())} if 0 in keep else {}
    h = dt_rk
    for k in range(1, n_steps + 1):
        k1u, k1v = v, acc(u)
        k2u, k2v = v + 0.5 * h * k1v, acc(u + 0.5 * h * k1u)
        k3u, k3v = v + 0.5 * h * k2v, acc(u + 0.5 * h * k2u)
        k4u, k4v = v + h * k3v, acc(u + h * k3u)
        u = u + h / 6.0 * (k1u + 2 * k2u + 2 * k3u + k4u)
        v = v + h / 6.0 * (k1v + 2 * k2v + 2 * k3v + k4v)
        if k in keep:
            out[k] = (u.copy(), v.copy())
    return out


def _smooth_nh_beam():
    return inputs.beam_neohooke(nel=(8, 2, 2), dt=0.1, steps=0, jitter=False)


def test_nonlinear_converges_to_split_independent_rk4():
    """Section 3 (Eq. "timeDiscError") and Section 4.2: the midpoint propagator with the secant
    split converges at second order to the solution of M u'' = -R(u), whose limit does not
    depend on how H(u) is split. A wrong split (H(u*) u* != R(u*)), a wrong midpoint or a wrong
    mass scaling would converge to something else, or not at second order."""
    prob = _smooth_nh_beam()
    T, dt_rk = 1.0, 0.0005
    n = int(round(T / dt_rk))
    u_ref, v_ref = _rk4_reference(prob, dt_rk, n)[n]
    errs = []
    for dt in (0.05, 0.025, 0.0125):
        P = propagator.Propagator.from_problem(prob)
        for _ in range(int(round(T / dt))):
            P.step(dt, 1e-13)
        fe = P.fe
        u, v = P.u_full()[fe.free], P.v_full()[fe.free]
        errs.append([np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref),
                     np.linalg.norm(v - v_ref) / np.linalg.norm(v_ref)])
    errs = np.array(errs)
    slopes = np.log(errs[:-1] / errs[1:]) / np.log(2.0)
    assert np.all(slopes > 1.8), (errs, slopes)
    assert errs[-1, 0] < 5e-6 and errs[-1, 1] < 1e-3, errs


@pytest.mark.parametrize("variant", ["paper", "swapped", "constant"])
def test_predictor_local_order_with_exact_history(variant):
    """Section 4.2: the predictor extrapolates the two previous midpoint operators linearly to
    t_{n-1} + dt/4 (weights 1.75 on H(u_{n-3/2}), -0.75 on H(u_{n-5/2})), so with exact history
    its half-step displacement u_{n-1/2} has a local error of O(dt^4) (exponential midpoint
    rule with an O(dt^2) operator). The history slots are filled from the RK4 reference and the
    oracle's own step is run: wrong weights or swapped slots (an O(dt) operator error) give
    O(dt^3) and errors 30-100x larger at dt = 0.01, which the bounds below reject; the
    "swapped" and "constant" cases plant those mistakes in the history to show it."""
    prob = _smooth_nh_beam()
    dt_rk, t0 = 0.00025, 0.3
    n0 = int(round(t0 / dt_rk))
    dts = (0.04, 0.02, 0.01)
    keep = {n0}
    for dt in dts:
        h = int(round(0.5 * dt / dt_rk))
        keep |= {n0 - 3 * h, n0 - h, n0 + h}
    ref = _rk4_reference(prob, dt_rk, n0 + max(keep) - n0, keep)
    errs = []
    for dt in dts:
        P = propagator.Propagator.from_problem(prob)
        fe = P.fe
        h = int(round(0.5 * dt / dt_rk))
        u, v = ref[n0]
        P.w = np.concatenate([P.sqm * u, P.sqm * v])
        older, newer = fe.to_full(ref[n0 - 3 * h][0]), fe.to_full(ref[n0 - h][0])
        P.mid_history = {"paper": [older, newer], "swapped": [newer, older],
                         "constant": [newer, newer]}[variant]
        P.step(dt, 1e-13)
        u_half = P.mid_history[-1][fe.free]  # the predictor's u_{n-1/2}
        u_ex = ref[n0 + h][0]
        errs.append(np.linalg.norm(u_half - u_ex) / np.linalg.norm(u_ex))
    errs = np.array(errs)
    slopes = np.log(errs[:-1] / errs[1:]) / np.log(2.0)
    ok = bool(np.all(slopes > 3.5) and errs[-1] < 1e-7)
    assert ok == (variant == "paper"), (variant, errs, slopes)


def test_newmark_linear_energy_and_order():
    p = inputs.beam_linear()
    N = Newmark.from_problem(p)
    E0 = N.energy()[0]
    for _ in range(50):
        N.step(0.05)
    assert abs(N.energy()[0] - E0) / E0 < 1e-10  # trapezoidal rule conserves energy
    # second order against the exact modal solution
    P = propagator.Propagator.from_problem(p)
    w0 = P.w.copy()
    ub, _ = _modal(P, w0, 0.2)
    u_ex = P.fe.to_full(ub / P.sqm)
    errs = []
    for dt in [0.004, 0.002, 0.001]:
        N = Newmark.from_problem(p)
        for _ in range(int(round(0.2 / dt))):
            N.step(dt)
        errs.append(np.linalg.norm(N.fe.to_full(N.u) - u_ex) / np.linalg.norm(u_ex))
    slopes = np.log(np.array(errs[:-1]) / np.array(errs[1:])) / np.log(2)
    assert np.all((slopes > 1.8) & (slopes < 2.2)), slopes


def test_tangent_is_derivative_of_force():
    p = _small_nh_beam(0.1)
    P = propagator.Propagator.from_problem(p)
    fe = P.fe
    rng = np.random.default_rng(0)
    u = fe.to_full(0.05 * rng.standard_normal(fe.Nf))
    KT = fe.assemble_H(p.material, p.params, u, tangent=True)
    d = rng.standard_normal(fe.Nf)
    h = 1e-6
    fd = (fe.internal_force(p.material, p.params, u + h * fe.to_full(d))
          - fe.internal_force(p.material, p.params, u - h * fe.to_full(d)))[fe.free] / (2 * h)
    np.testing.assert_allclose(KT @ d, fd, atol=1e-6 * np.abs(fd).max())


def test_newmark_nonlinear_agrees_with_exponential():
    """Both integrators are second order; at a small dt they agree to O(dt^2)."""
    p = _small_nh_beam(0.01)
    N = Newmark.from_problem(p)
    P = propagator.Propagator.from_problem(p)
    for _ in range(100):
        N.step(0.01)
        P.step(0.01, 1e-12)
    u_n, u_p = N.fe.to_full(N.u), P.u_full()
    assert np.linalg.norm(u_n - u_p) <= 1e-3 * np.linalg.norm(u_p)
