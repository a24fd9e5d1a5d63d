"""The persistent step's norm reading, checked on the CPU (no GPU).

The GPU's short-vector Arnoldi step takes the subdiagonal entry from the second CGS pass,
h_{j+1,j}^2 = ||z'||^2 - sum_i h2_i^2 (z' the vector after the first pass, h2 its coefficients), and
sums ||z''||^2 directly only where that difference falls below 1/16 of ||z'||^2. In exact arithmetic
the two are equal when V is orthonormal (Section 4.3's Arnoldi relation with CGS2). These tests run
both forms side by side in numpy on the same inputs and compare them with the oracle's CGS2
(`oracle/krylov.py`, direct norm): the Hessenberg matrices agree to rounding, the FP32-basis form to
FP32 rounding, and near a breakdown the fallback is the branch taken.
"""
import numpy as np

from oracle import krylov


def _arnoldi_pythagorean(A, w, m, basis_dtype=np.float64):
    """CGS2 Arnoldi whose subdiagonal comes from the second pass; basis stored in basis_dtype,
    sums in FP64. Returns H and the list of steps that took the direct-norm fallback."""
    L = w.size
    V = np.zeros((L, m + 1), dtype=basis_dtype)
    H = np.zeros((m + 1, m))
    V[:, 0] = (w / np.linalg.norm(w)).astype(basis_dtype)
    fallback = []
    for j in range(m):
        Vj = V[:, : j + 1].astype(np.float64)
        z = (A @ Vj[:, j]).astype(basis_dtype).astype(np.float64)
        h1 = Vj.T @ z
        z1 = (z - Vj @ h1).astype(basis_dtype).astype(np.float64)
        h2 = Vj.T @ z1
        n1 = float(z1 @ z1)
        z2 = (z1 - Vj @ h2).astype(basis_dtype)
        H[: j + 1, j] = h1 + h2
        n2 = n1 - float(h2 @ h2)
        if not (n2 > n1 / 16.0):
            n2 = float(z2.astype(np.float64) @ z2.astype(np.float64))
            fallback.append(j)
        hn = np.sqrt(n2)
        H[j + 1, j] = hn
        if hn <= 1e-14 * np.linalg.norm(H[: j + 1, : j + 1]):
            return H[: j + 2, : j + 1], fallback, True
        V[:, j + 1] = (z2.astype(np.float64) / hn).astype(basis_dtype)
    return H, fallback, False


def _oracle_H(A, w, m):
    r = krylov.arnoldi_expv(lambda x: A @ x, w, 1.0, 0.0, m, m_fixed=m, keep_basis=True)
    return r.H


def _problem(n=300, seed=5):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    w = rng.standard_normal(n)
    return A, w


def test_pythagorean_subdiagonal_equals_direct_cgs2_in_fp64():
    A, w = _problem()
    m = 40
    Hp, fallback, _ = _arnoldi_pythagorean(A, w, m)
    Ho = _oracle_H(A, w, m)
    assert not fallback  # a well-conditioned process never cancels
    assert np.max(np.abs(Hp - Ho)) / np.max(np.abs(Ho)) < 1e-13
    sub_p, sub_o = np.diag(Hp, -1), np.diag(Ho, -1)
    assert np.max(np.abs(sub_p - sub_o) / sub_o) < 1e-12


def test_pythagorean_subdiagonal_with_an_fp32_basis():
    """FP32 basis and vectors, FP64 sums (the MIXED form): the subdiagonal matches the direct norm of
    the stored FP32 vector to FP32 rounding, and H the oracle's to the FP32 level."""
    A, w = _problem(seed=9)
    m = 30
    Hp, fallback, _ = _arnoldi_pythagorean(A, w, m, basis_dtype=np.float32)
    Ho = _oracle_H(A, w, m)
    assert not fallback
    assert np.max(np.abs(Hp - Ho)) / np.max(np.abs(Ho)) < 1e-5


def test_fallback_at_a_breakdown():
    """w in an exactly invariant 6-dimensional subspace (a diagonal operator, w on 6 coordinates: the
    other coordinates stay exactly zero). At the 6th step z' is rounding noise inside span(V), so
    the second pass removes all of it, the difference cancels, the direct norm is taken, and the
    breakdown is seen at the same step as in the oracle."""
    rng = np.random.default_rng(11)
    n, k = 200, 6
    A = np.diag(np.concatenate([np.linspace(1.0, 2.0, k), rng.uniform(3.0, 4.0, n - k)]))
    w = np.zeros(n)
    w[:k] = rng.standard_normal(k)
    Hp, fallback, broke = _arnoldi_pythagorean(A, w, 20)
    r = krylov.arnoldi_expv(lambda x: A @ x, w, 1.0, 0.0, 20, m_fixed=20, keep_basis=True)
    assert broke and r.breakdown
    assert Hp.shape[1] == r.m == k
    assert fallback == [k - 1]
    assert np.max(np.abs(Hp[:k, :k] - r.H[:k, :k])) < 1e-12
