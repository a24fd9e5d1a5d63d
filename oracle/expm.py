"""Dense matrix exponentials for the small Hessenberg matrix, FP64 (test infrastructure).

Section 4.3 of arXiv 2405.05213 evaluates ``exp(H_m)`` by a Taylor series when
``||H_m|| <= 1`` and by scaling and squaring otherwise, never by an
eigendecomposition (H_m is non-normal).

``expm_pade`` is the scaling-and-squaring algorithm with the diagonal [13/13]
Pade approximant (Higham, SIAM J. Matrix Anal. Appl. 26 (2005) 1179-1193):
scale by 2^-s so that ||A||_1 <= theta_13, evaluate r_13 = q(A)^-1 p(A), square
s times. The Pade coefficients come from their closed form
``c_k = (2m-k)! m! / ((2m)! k! (m-k)!)`` with m = 13, computed exactly.

``expm_taylor`` is the paper's "direct exponentiation": the Taylor series
summed until the terms stop changing the sum, after scaling so the series is
well conditioned, then squared back.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

PADE_M = 13
THETA_13 = 5.371920351148152  # Higham 2005, Table 2.3, m = 13


def pade_coefficients(m: int = PADE_M) -> np.ndarray:
    """c_k of the numerator p(x) = sum_k c_k x^k of the [m/m] Pade approximant of e^x."""
    c = [Fraction(math.factorial(2 * m - k) * math.factorial(m),
                  math.factorial(2 * m) * math.factorial(k) * math.factorial(m - k))
         for k in range(m + 1)]
    return np.array([float(x) for x in c])


_C13 = pade_coefficients(13)


def expm_pade(A: np.ndarray) -> np.ndarray:
    """exp(A) by Pade [13/13] scaling and squaring."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if n == 0:
        return np.zeros((0, 0))
    nrm = np.abs(A).sum(axis=0).max()
    s = 0
    if nrm > THETA_13:
        s = int(math.ceil(math.log2(nrm / THETA_13)))
    B = A / (2.0 ** s)
    I = np.eye(n)
    B2 = B @ B
    B4 = B2 @ B2
    B6 = B4 @ B2
    c = _C13
    # odd part U = B (B6 (c13 B6 + c11 B4 + c9 B2) + c7 B6 + c5 B4 + c3 B2 + c1 I)
    U = B @ (B6 @ (c[13] * B6 + c[11] * B4 + c[9] * B2) + c[7] * B6 + c[5] * B4 + c[3] * B2 + c[1] * I)
    # even part V = B6 (c12 B6 + c10 B4 + c8 B2) + c6 B6 + c4 B4 + c2 B2 + c0 I
    V = B6 @ (c[12] * B6 + c[10] * B4 + c[8] * B2) + c[6] * B6 + c[4] * B4 + c[2] * B2 + c[0] * I
    R = np.linalg.solve(V - U, V + U)  # q(B) = p(-B) = V - U, p(B) = V + U
    for _ in range(s):
        R = R @ R
    return R


def expm_taylor(A: np.ndarray, scale_to: float = 0.5) -> np.ndarray:
    """exp(A) by a Taylor series to machine precision after scaling by 2^-s."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    nrm = np.abs(A).sum(axis=0).max() if n else 0.0
    s = 0
    if nrm > scale_to:
        s = int(math.ceil(math.log2(nrm / scale_to)))
    B = A / (2.0 ** s)
    E = np.eye(n)
    term = np.eye(n)
    for k in range(1, 60):
        term = term @ B / k
        E_new = E + term
        if np.array_equal(E_new, E):
            break
        E = E_new
    for _ in range(s):
        E = E @ E
    return E
