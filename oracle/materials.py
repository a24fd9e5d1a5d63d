"""Hyperelastic constitutive laws and their secant (H-matrix) split, FP64.

Test infrastructure: imported only by the tests, ``smoke()`` and the bench's
CPU-baseline leg.

All functions act on batches of 3x3 tensors of shape (..., 3, 3).

Passages of arXiv 2405.05213 followed:

* Section 2.1, Eq. "Constitutive equation": ``S = d psi / dE``,
  ``E = (F^T F - I)/2``, ``F = I + grad u``.
* Appendix A.1: St. Venant-Kirchhoff, ``psi = lambda/2 (tr E)^2 + mu tr(E^2)``,
  ``S = lambda tr(E) I + 2 mu E``.
* Appendix A.2: Yeoh, ``psi = C10 (I1b-3) + C20 (I1b-3)^2 + C30 (I1b-3)^3 +
  (J-1)^2 / D1`` and its S with the frozen scalars alpha_e, beta_e, plus the
  matrix P_e with ``det F - 1 = P_e : grad u`` (the "detF - 1" identity).
* Appendix A, opening paragraph: Neo-Hookean and Mooney-Rivlin follow the same
  construction (the paper gives no formulas; the readings below are ours).

The secant split (Section 2.3, ``R(u) = H(u) u``) is not unique. The reading
used on both sides of the parity check is the frozen-coefficient secant:
with ``D* = grad u*``, ``F* = I + D*``, ``C* = F*^T F*``, ``J* = det F*`` and a
linear argument ``G``:

* ``E_lin(G) = sym(G) + sym(D*^T G) / 2``, so ``E_lin(D*) = E*``;
* ``j_lin(G) = P_e(D*) : G`` with ``P_e(D) = I + (tr D I - D^T)/2 + cof(D)/3``,
  so ``j_lin(D*) = J* - 1`` exactly;
* ``P_lin(G) = F* S_lin(G)`` where ``S_lin`` is the stress with every nonlinear
  coefficient frozen at u*, chosen so that ``S_lin(D*) = S(E*)``; hence
  ``P_lin(D*) = P(F*)`` and ``H(u*) u* = R(u*)``.
"""
from __future__ import annotations

import numpy as np

LINEAR, NEOHOOKE, MOONEY_RIVLIN, SVK, YEOH = 0, 1, 2, 3, 4

_I = np.eye(3)


def _tr(A):
    return np.trace(A, axis1=-2, axis2=-1)


def _T(A):
    return np.swapaxes(A, -1, -2)


def _sym(A):
    return 0.5 * (A + _T(A))


def _ddot(A, B):
    return np.sum(A * B, axis=(-2, -1))


def _sc(s):
    """Broadcast a (...) scalar field against (..., 3, 3)."""
    return np.asarray(s)[..., None, None]


def cofactor(D):
    """Cofactor matrix: cof(D)_ij = (-1)^(i+j) times the (i, j) minor of D."""
    c = np.empty_like(D)
    for i in range(3):
        i1, i2 = (i + 1) % 3, (i + 2) % 3
        for j in range(3):
            j1, j2 = (j + 1) % 3, (j + 2) % 3
            c[..., i, j] = D[..., i1, j1] * D[..., i2, j2] - D[..., i1, j2] * D[..., i2, j1]
    return c


def P_e(D):
    """Appendix A.2 matrix with ``det(I + D) - 1 = P_e(D) : D``."""
    return _I + 0.5 * (_sc(_tr(D)) * _I - _T(D)) + cofactor(D) / 3.0


def log_ratio(J):
    """ln(J) / (J - 1), continuous at J = 1."""
    x = np.asarray(J) - 1.0
    small = np.abs(x) < 1e-8
    xs = np.where(small, 1.0, x)
    return np.where(small, 1.0 - x / 2.0 + x * x / 3.0, np.log1p(xs) / xs)


# ------------------------------------------------------------------ full laws
def pk2(kind, params, F):
    """Second Piola-Kirchhoff stress S(F) (for LINEAR: the small-strain stress)."""
    if kind == LINEAR:
        lam, mu = _lame(params)
        eps = _sym(F - _I)
        return lam * _sc(_tr(eps)) * _I + 2 * mu * eps
    C = _T(F) @ F
    J = np.linalg.det(F)
    Ci = np.linalg.inv(C)
    I1 = _tr(C)
    if kind == NEOHOOKE:
        mu, lam = params[0], params[1]
        return mu * (_I - Ci) + lam * _sc(np.log(J)) * Ci
    if kind == MOONEY_RIVLIN:
        c10, c01, kappa = params[0], params[1], params[2]
        I2 = 0.5 * (I1 ** 2 - _tr(C @ C))
        t1 = 2 * c10 * _sc(J ** (-2.0 / 3.0)) * (_I - _sc(I1 / 3.0) * Ci)
        t2 = 2 * c01 * _sc(J ** (-4.0 / 3.0)) * (_sc(I1) * _I - C - _sc(2.0 * I2 / 3.0) * Ci)
        t3 = kappa * _sc(J * (J - 1.0)) * Ci
        return t1 + t2 + t3
    if kind == SVK:
        lam, mu = params[0], params[1]
        E = 0.5 * (C - _I)
        return lam * _sc(_tr(E)) * _I + 2 * mu * E
    if kind == YEOH:
        c10, c20, c30, d1 = params[0], params[1], params[2], params[3]
        I1b = J ** (-2.0 / 3.0) * I1
        alpha = 2 * J ** (-2.0 / 3.0) * (c10 + 2 * c20 * (I1b - 3) + 3 * c30 * (I1b - 3) ** 2)
        return _sc(alpha) * (_I - _sc(I1 / 3.0) * Ci) + _sc(2.0 / d1 * J * (J - 1.0)) * Ci
    raise ValueError(kind)


def pk1(kind, params, F):
    """First Piola stress P = F S (LINEAR: the small-strain stress itself)."""
    S = pk2(kind, params, F)
    if kind == LINEAR:
        return S
    return F @ S


def psi(kind, params, F):
    """Strain energy density."""
    if kind == LINEAR:
        lam, mu = _lame(params)
        eps = _sym(F - _I)
        return 0.5 * lam * _tr(eps) ** 2 + mu * _ddot(eps, eps)
    C = _T(F) @ F
    J = np.linalg.det(F)
    I1 = _tr(C)
    if kind == NEOHOOKE:
        mu, lam = params[0], params[1]
        lnJ = np.log(J)
        return 0.5 * mu * (I1 - 3) - mu * lnJ + 0.5 * lam * lnJ ** 2
    if kind == MOONEY_RIVLIN:
        c10, c01, kappa = params[0], params[1], params[2]
        I2 = 0.5 * (I1 ** 2 - _tr(C @ C))
        return (c10 * (J ** (-2.0 / 3.0) * I1 - 3) + c01 * (J ** (-4.0 / 3.0) * I2 - 3)
                + 0.5 * kappa * (J - 1) ** 2)
    if kind == SVK:
        lam, mu = params[0], params[1]
        E = 0.5 * (C - _I)
        return 0.5 * lam * _tr(E) ** 2 + mu * _tr(E @ E)
    if kind == YEOH:
        c10, c20, c30, d1 = params[0], params[1], params[2], params[3]
        x = J ** (-2.0 / 3.0) * I1 - 3
        return c10 * x + c20 * x ** 2 + c30 * x ** 3 + (J - 1) ** 2 / d1
    raise ValueError(kind)


def _lame(params):
    E, nu = params[0], params[1]
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


# ------------------------------------------------------------------ secant split
def plin(kind, params, G, Dstar):
    """Secant first Piola stress P_lin(G; D*), linear in G, with P_lin(D*) = P(I + D*)."""
    if kind == LINEAR:
        lam, mu = _lame(params)
        eps = _sym(G)
        return lam * _sc(_tr(eps)) * _I + 2 * mu * eps
    if Dstar is None:
        Dstar = np.zeros_like(G)
    Dstar = np.broadcast_to(Dstar, G.shape)
    F = _I + Dstar
    C = _T(F) @ F
    Ci = np.linalg.inv(C)
    J = np.linalg.det(F)
    Es = 0.5 * (C - _I)
    El = _sym(G) + 0.5 * _sym(_T(Dstar) @ G)
    jl = _ddot(P_e(Dstar), G)
    if kind == NEOHOOKE:
        mu, lam = params[0], params[1]
        S = 2 * mu * _sym(Ci @ El) + lam * _sc(log_ratio(J) * jl) * Ci
    elif kind == MOONEY_RIVLIN:
        c10, c01, kappa = params[0], params[1], params[2]
        es, el = _tr(Es), _tr(El)
        dev2El = 2 * El - _sc(2.0 * el / 3.0) * _I
        Q = (2 * El - _sc(2.0 * el / 3.0) * _I
             + 2 * (_sc(es) * El + _sc(el) * Es)
             - 2 * (Es @ El + El @ Es)
             - _sc(4.0 / 3.0 * (es * el - _ddot(Es, El))) * _I)
        S = (2 * c10 * _sc(J ** (-2.0 / 3.0)) * _sym(Ci @ dev2El)
             + 2 * c01 * _sc(J ** (-4.0 / 3.0)) * _sym(Q @ Ci)
             + kappa * _sc(J * jl) * Ci)
    elif kind == SVK:
        lam, mu = params[0], params[1]
        S = lam * _sc(_tr(El)) * _I + 2 * mu * El
    elif kind == YEOH:
        c10, c20, c30, d1 = params[0], params[1], params[2], params[3]
        I1b = J ** (-2.0 / 3.0) * _tr(C)
        alpha = 2 * J ** (-2.0 / 3.0) * (c10 + 2 * c20 * (I1b - 3) + 3 * c30 * (I1b - 3) ** 2)
        beta = 2.0 / d1 * J
        dev2El = 2 * El - _sc(2.0 * _tr(El) / 3.0) * _I
        S = _sc(alpha) * _sym(Ci @ dev2El) + _sc(beta * jl) * Ci
    else:
        raise ValueError(kind)
    return F @ S
