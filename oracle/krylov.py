"""Arnoldi/Krylov evaluation of exp(tau A) w, FP64 (test infrastructure).

Section 4.3 of arXiv 2405.05213:

* the Krylov basis V_m with ``v_1 = w / ||w||`` and the upper Hessenberg H_m
  satisfy ``A V_m = V_m H_m + h_{m+1,m} v_{m+1} e_m^T`` (Arnoldi relation);
* ``exp(tau A) w ~= ||w|| V_m exp(tau H_m) e_1``;
* Eq. "subspace error estimate": with ``tau`` folded into the operator,
  ``eps_m = tau h_{m+1,m} ||w|| |[exp(tau H_m)]_{m,1}|``; the subspace size is
  the smallest m whose estimate meets the tolerance. The tolerance is read as
  relative: stop when ``eps_m <= tol ||w||``.

Orthogonalisation is classical Gram-Schmidt with one full reorthogonalisation
pass (CGS2): ``h = V^T z; z -= V h`` twice, coefficients summed.
A happy breakdown (``h_{m+1,m} <= 1e-14 ||H_m||_F``) ends the process with the
exact result.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .expm import expm_pade


@dataclass
class KrylovResult:
    w: np.ndarray
    m: int
    eps: float
    converged: bool
    breakdown: bool
    V: np.ndarray | None = None
    H: np.ndarray | None = None


def arnoldi_expv(apply, w, tau, tol, m_cap, m_fixed=0, keep_basis=False, expm=expm_pade):
    """exp(tau A) w with the a-priori estimate choosing m (or m = m_fixed)."""
    w = np.asarray(w, dtype=np.float64)
    L = w.size
    beta = float(np.linalg.norm(w))
    if beta == 0.0:
        return KrylovResult(np.zeros(L), 0, 0.0, True, True)
    cap = m_fixed if m_fixed > 0 else m_cap
    V = np.zeros((L, cap + 1))
    H = np.zeros((cap + 1, cap))
    V[:, 0] = w / beta
    m, eps, converged, breakdown, E = 0, np.inf, False, False, None
    for j in range(cap):
        z = apply(V[:, j])
        Vj = V[:, : j + 1]
        h1 = Vj.T @ z
        z = z - Vj @ h1
        h2 = Vj.T @ z
        z = z - Vj @ h2
        H[: j + 1, j] = h1 + h2
        hn = float(np.linalg.norm(z))
        H[j + 1, j] = hn
        m = j + 1
        breakdown = hn <= 1e-14 * np.linalg.norm(H[:m, :m])
        if not breakdown:
            V[:, j + 1] = z / hn
        last = breakdown or m == cap
        if m_fixed == 0 or last:
            E = expm(tau * H[:m, :m])
            eps = 0.0 if breakdown else beta * tau * hn * abs(E[m - 1, 0])
            if breakdown or (m_fixed == 0 and eps <= tol * beta):
                converged = True
                break
            if last:
                converged = m_fixed > 0
                break
    y = beta * E[:, 0]
    w_new = V[:, :m] @ y
    res = KrylovResult(w_new, m, float(eps), converged, breakdown)
    if keep_basis:
        res.V, res.H = V[:, : m + 1], H[: m + 1, :m]
    return res
