"""Pins for the oracle's small exponential and Arnoldi process (no GPU)."""
import os

import numpy as np
import pytest
import scipy.linalg

import inputs
from oracle import expm as oexpm
from oracle import krylov, propagator


def test_pade_coefficients_match_higham_table(root):
    vals = [int(l) for l in open(os.path.join(root, "tests", "golden", "pade13_higham2005.txt"))
            if l.strip() and not l.startswith("#")]
    c = oexpm.pade_coefficients(13)
    b = np.array(vals, dtype=np.float64)
    np.testing.assert_allclose(c / c[13], b, rtol=1e-15)
    assert c[0] == 1.0 and c[1] == 0.5


def test_scalar_pade_is_exp():
    c = oexpm.pade_coefficients(13)
    for x in np.linspace(-oexpm.THETA_13, oexpm.THETA_13, 11):
        p = np.polyval(c[::-1], x)
        q = np.polyval(c[::-1], -x)
        assert abs(p / q - np.exp(x)) < 4e-16 * np.exp(x) * 8


@pytest.mark.parametrize("expm", [oexpm.expm_pade, oexpm.expm_taylor])
def test_expm_closed_forms(expm):
    for th in [0.1, 1.0, 7.5, 40.0]:
        A = np.array([[0.0, th], [-th, 0.0]])
        R = np.array([[np.cos(th), np.sin(th)], [-np.sin(th), np.cos(th)]])
        np.testing.assert_allclose(expm(A), R, atol=2e-14 * max(1, th))
    np.testing.assert_array_equal(expm(np.zeros((4, 4))), np.eye(4))
    N = np.triu(np.ones((4, 4)), 1)  # nilpotent: exp = I + N + N^2/2 + N^3/6
    np.testing.assert_allclose(expm(N), np.eye(4) + N + N @ N / 2 + N @ N @ N / 6, atol=1e-15)
    d = np.array([-3.0, 0.5, 2.0, 9.0])
    np.testing.assert_allclose(expm(np.diag(d)), np.diag(np.exp(d)), rtol=5e-14)


@pytest.mark.parametrize("expm", [oexpm.expm_pade, oexpm.expm_taylor])
def test_expm_against_library(expm):
    rng = np.random.default_rng(0)
    for n, scale in [(5, 0.1), (20, 2.0), (40, 10.0), (64, 30.0)]:
        A = np.triu(rng.standard_normal((n, n)), -1) * scale / np.sqrt(n)  # upper Hessenberg
        ref = scipy.linalg.expm(A)
        np.testing.assert_allclose(expm(A), ref, atol=1e-12 * np.abs(ref).max())
        E = expm(A) @ expm(-A)
        assert np.abs(E - np.eye(n)).max() < 1e-9 * max(1.0, np.abs(ref).max())


def _beam_linear_operator():
    p = inputs.beam_linear()
    P = propagator.Propagator.from_problem(p)
    Hb = P.Hbar(None)
    Nf = P.Nf
    A = np.block([[np.zeros((Nf, Nf)), np.eye(Nf)], [-Hb.toarray(), np.zeros((Nf, Nf))]])
    return p, P, A


def test_arnoldi_relation_and_orthogonality():
    p, P, A = _beam_linear_operator()
    r = krylov.arnoldi_expv(P.A_apply(P.Hbar(None)), P.w, p.dt, 1e-12, 60, keep_basis=True)
    V, H = r.V, r.H
    m = r.m
    nA = np.linalg.norm(A, 2)
    res = A @ V[:, :m] - V @ H
    assert np.linalg.norm(res) / nA < 1e-13
    assert np.abs(V.T @ V - np.eye(m + 1)).max() < 1e-13


def test_krylov_vs_dense_exponential():
    """The paper's own check: Krylov result vs direct exponentiation (Section 6.1)."""
    p, P, A = _beam_linear_operator()
    rng = np.random.default_rng(1)
    w = P.w + 1e-3 * rng.standard_normal(P.w.size)
    nw = np.linalg.norm(w)
    ratios = []
    for dt in [0.01, 0.05, 0.2]:
        ref = scipy.linalg.expm(dt * A) @ w
        for m in range(4, 60, 4):
            r = krylov.arnoldi_expv(P.A_apply(P.Hbar(None)), w, dt, 0.0, 200, m_fixed=m)
            err = np.linalg.norm(r.w - ref) / nw
            # asymptotic regime, above the dense reference's own rounding floor
            if 1e-10 < err < 1e-2:
                ratios.append(r.eps / nw / err)
        r = krylov.arnoldi_expv(P.A_apply(P.Hbar(None)), w, dt, 1e-10, 200)
        assert r.converged
        assert np.linalg.norm(r.w - ref) <= 1e-9 * np.linalg.norm(ref)
    # the estimate traces the true error once the subspace converges (Section 6.1)
    ratios = np.array(ratios)
    assert len(ratios) >= 6
    assert np.all((ratios > 0.3) & (ratios < 10.0)), ratios


def test_happy_breakdown_is_exact():
    n = 30
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    D = np.diag(np.r_[np.arange(1.0, 4.0), np.zeros(n - 3)])
    A = Q @ D @ Q.T
    w = Q[:, :3] @ np.array([1.0, -2.0, 0.5])  # lies in a 3-dim invariant subspace
    r = krylov.arnoldi_expv(lambda x: A @ x, w, 0.7, 1e-14, 20)
    assert r.breakdown and r.m == 3
    np.testing.assert_allclose(r.w, scipy.linalg.expm(0.7 * A) @ w, atol=1e-13)
