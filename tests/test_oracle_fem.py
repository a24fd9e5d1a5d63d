"""Pins for the oracle's discretisation and constitutive laws (no GPU).

Each test checks the oracle against something other than itself: textbook
quadrature tables, closed forms, invariants, or finite differences of an
independently written quantity.
"""
import os

import numpy as np
import pytest

import inputs
from oracle import fem, materials

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

ALL_KINDS = [
    (materials.LINEAR, (1.0e3, 0.3)),
    (materials.NEOHOOKE, (345.0, 805.0)),
    (materials.MOONEY_RIVLIN, (0.5, 0.05, 1.1e3)),
    (materials.SVK, (805.0, 345.0)),
    (materials.YEOH, (100.0, -1.0, 0.01, 0.001)),
]
NONLINEAR = ALL_KINDS[1:]


def _golden(root, name):
    return os.path.join(root, "tests", "golden", name)


def test_quadrature_matches_tables(root):
    for line in open(_golden(root, "quadrature_abramowitz_stegun.txt")):
        if line.startswith("#") or not line.strip():
            continue
        head, w = line.split("|")
        parts = head.split()
        rule, n, pts = parts[0], int(parts[1]), np.array(parts[2:], float)
        w = np.array(w.split(), float)
        p, ww = fem.gauss_legendre(n) if rule == "gauss" else fem.gll(n)
        np.testing.assert_allclose(p, pts, atol=1e-15)
        np.testing.assert_allclose(ww, w, atol=1e-15)


@pytest.mark.parametrize("n", [2, 3])
def test_gauss_exact_to_degree(n):
    p, w = fem.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * p ** k) - exact) < 1e-14


@pytest.mark.parametrize("order", [1, 2])
def test_shape_functions_basic(order):
    xi = np.linspace(-1, 1, 7)
    N, dN = fem.lagrange_1d(order, xi)
    np.testing.assert_allclose(N.sum(axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(dN.sum(axis=1), 0.0, atol=1e-14)
    Nn, _ = fem.lagrange_1d(order, fem.lagrange_nodes(order))
    np.testing.assert_allclose(Nn, np.eye(order + 1), atol=1e-15)
    # derivative vs central differences
    h = 1e-6
    Np, _ = fem.lagrange_1d(order, xi + h)
    Nm, _ = fem.lagrange_1d(order, xi - h)
    np.testing.assert_allclose((Np - Nm) / (2 * h), dN, atol=1e-8)
    p, w = fem.gauss_legendre(order + 1)
    N3, dN3, w3 = fem.shape_3d(order, p, w)
    np.testing.assert_allclose(N3.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(dN3.sum(axis=1), 0.0, atol=1e-13)
    assert abs(w3.sum() - 8.0) < 1e-13


def _disc(mesh, fixed=None, rho=1.0):
    fixed = np.zeros(0, np.int32) if fixed is None else fixed
    return fem.Discretisation(mesh.order, mesh.coords, mesh.conn, fixed, rho)


@pytest.mark.parametrize("order", [1, 2])
def test_mass_total_and_rowsum_lumping(order):
    mesh = inputs.box_mesh(order, 3, 2, 2, 1.5, 1.0, 0.8)
    d = _disc(mesh, rho=2.5)
    assert abs(d.mass[0::3].sum() - 2.5 * 1.5 * 1.0 * 0.8) < 1e-12
    # consistent mass by Gauss quadrature, then row sums (affine elements)
    p, w = fem.gauss_legendre(order + 2)
    Nq, _, wq = fem.shape_3d(order, p, w)
    X = mesh.coords[mesh.conn]
    _, dNq, _ = fem.shape_3d(order, p, w)
    J = np.einsum("eai,qaj->eqij", X, dNq)
    dV = np.linalg.det(J) * wq
    Me = np.einsum("qa,qb,eq->eab", Nq, Nq, 2.5 * dV)
    rows = np.zeros(mesh.n_nodes)
    np.add.at(rows, mesh.conn.ravel(), Me.sum(axis=2).ravel())
    np.testing.assert_allclose(d.mass[0::3], rows, rtol=1e-13)
    # perturbed mesh: total still rho * volume
    pm = inputs.perturb_interior(mesh, 7)
    assert abs(_disc(pm).mass[0::3].sum() - 1.5 * 1.0 * 0.8) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_stiffness_rigid_modes(order):
    mesh = inputs.perturb_interior(inputs.box_mesh(order, 3, 2, 2, 2.0, 1.0, 1.0), 3)
    d = _disc(mesh)
    K = d.assemble_H(materials.LINEAR, (1.0, 0.3), None)
    X = mesh.coords
    nrmK = abs(K).sum(axis=1).max()
    for c in range(3):
        t = np.zeros((mesh.n_nodes, 3))
        t[:, c] = 1.0
        assert np.abs(K @ t.ravel()).max() < 1e-12 * nrmK
    for (a, b) in [(0, 1), (1, 2), (0, 2)]:
        r = np.zeros((mesh.n_nodes, 3))
        r[:, a] = -X[:, b]
        r[:, b] = X[:, a]
        assert np.abs(K @ r.ravel()).max() < 1e-12 * nrmK * X.max()
    # symmetric positive semi-definite with exactly six zero modes
    Kd = K.toarray()
    np.testing.assert_allclose(Kd, Kd.T, atol=1e-12 * nrmK)
    ev = np.linalg.eigvalsh(Kd)
    assert np.sum(ev < 1e-10 * ev[-1]) == 6


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("kind,params", ALL_KINDS)
def test_patch_test(order, kind, params):
    """A homogeneous deformation gives zero internal force at interior nodes."""
    mesh = inputs.perturb_interior(inputs.box_mesh(order, 3, 3, 2, 1.0, 1.0, 1.0), 11)
    d = _disc(mesh)
    B = np.array([[0.02, 0.01, -0.005], [0.003, -0.01, 0.004], [0.0, 0.006, 0.015]])
    u = (mesh.coords @ B.T).ravel()
    R = d.internal_force(kind, params, u).reshape(-1, 3)
    X = mesh.coords
    inner = np.all((X > 1e-9) & (X < 1 - 1e-9), axis=1)
    scale = np.abs(R).max()
    assert np.abs(R[inner]).max() < 1e-11 * scale


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("kind,params", ALL_KINDS)
def test_internal_force_is_energy_gradient(order, kind, params):
    mesh = inputs.perturb_interior(inputs.box_mesh(order, 2, 1, 1, 1.0, 0.5, 0.5), 5)
    d = _disc(mesh)
    rng = np.random.default_rng(0)
    u = 0.02 * rng.standard_normal(d.N)
    R = d.internal_force(kind, params, u)
    h = 1e-6
    for idx in rng.choice(d.N, 8, replace=False):
        e = np.zeros(d.N)
        e[idx] = h
        fd = (d.strain_energy(kind, params, u + e) - d.strain_energy(kind, params, u - e)) / (2 * h)
        assert abs(fd - R[idx]) <= 1e-6 * np.abs(R).max() + 1e-10


@pytest.mark.parametrize("kind,params", NONLINEAR)
def test_pk2_is_derivative_of_psi(kind, params):
    """S = 2 dpsi/dC, by central differences in C = F^T F through F = U (stretch)."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        D = 0.1 * rng.standard_normal((3, 3))
        F = np.eye(3) + D
        S = materials.pk2(kind, params, F)
        # dpsi along dF: dpsi = P : dF with P = F S
        P = F @ S
        h = 1e-6
        for _ in range(4):
            dF = rng.standard_normal((3, 3))
            fd = (materials.psi(kind, params, F + h * dF) - materials.psi(kind, params, F - h * dF)) / (2 * h)
            assert abs(fd - np.sum(P * dF)) < 1e-6 * max(1.0, np.abs(P).max())
        np.testing.assert_allclose(S, S.T, atol=1e-12 * np.abs(S).max())


@pytest.mark.parametrize("kind,params", ALL_KINDS)
def test_small_strain_limit_matches_lame(kind, params):
    """Linearisation at F = I gives lambda tr(eps) I + 2 mu eps with the recipe's moduli."""
    lam, mu = inputs.small_strain_moduli(kind, params)
    rng = np.random.default_rng(2)
    G = rng.standard_normal((3, 3))
    eps = 1e-7
    P = materials.pk1(kind, params, np.eye(3) + eps * G) / eps
    sym = 0.5 * (G + G.T)
    expect = lam * np.trace(sym) * np.eye(3) + 2 * mu * sym
    np.testing.assert_allclose(P, expect, rtol=0, atol=1e-5 * np.abs(expect).max())


def test_Pe_identity_and_cofactor():
    rng = np.random.default_rng(3)
    D = 0.3 * rng.standard_normal((20, 3, 3))
    lhs = np.linalg.det(np.eye(3) + D) - 1
    rhs = np.sum(materials.P_e(D) * D, axis=(-2, -1))
    np.testing.assert_allclose(lhs, rhs, atol=1e-14)
    cof = materials.cofactor(D)
    np.testing.assert_allclose(cof, np.linalg.det(D)[:, None, None] * np.linalg.inv(D).transpose(0, 2, 1), atol=1e-12)


def test_log_ratio():
    J = np.array([1.0, 1 + 1e-12, 1 - 1e-9, 1.3, 0.7])
    expect = np.array([1.0, 1.0 - 0.5e-12, 1.0 + 0.5e-9, np.log(1.3) / 0.3, np.log(0.7) / -0.3])
    np.testing.assert_allclose(materials.log_ratio(J), expect, rtol=1e-12)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("kind,params", NONLINEAR)
def test_split_reproduces_internal_force(order, kind, params):
    """H(u*) u* = R(u*) (Section 2.3) and H(0) = K."""
    mesh = inputs.perturb_interior(inputs.box_mesh(order, 2, 2, 1, 1.0, 1.0, 0.5), 9)
    fixed = inputs.fixed_dofs_on_plane(mesh, 0, 0.0)
    d = fem.Discretisation(order, mesh.coords, mesh.conn, fixed)
    rng = np.random.default_rng(4)
    u = d.to_full((0.05 if order == 1 else 0.01) * rng.standard_normal(d.Nf))
    H = d.assemble_H(kind, params, u)
    R = d.internal_force(kind, params, u)[d.free]
    assert np.all(np.isfinite(R))
    np.testing.assert_allclose(H @ u[d.free], R, atol=1e-12 * np.abs(R).max())
    lam, mu = inputs.small_strain_moduli(kind, params)
    E = mu * (3 * lam + 2 * mu) / (lam + mu)
    nu = lam / (2 * (lam + mu))
    K = d.assemble_H(materials.LINEAR, (E, nu), None)
    H0 = d.assemble_H(kind, params, np.zeros(d.N))
    np.testing.assert_allclose(H0.toarray(), K.toarray(), atol=1e-10 * abs(K).max())


def test_apply_at_nodes_matches_assembled():
    mesh = inputs.perturb_interior(inputs.box_mesh(2, 2, 2, 2, 1.0, 1.0, 1.0), 2)
    d = _disc(mesh)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(d.N)
    u = 0.03 * rng.standard_normal(d.N)
    H = d.assemble_H(materials.NEOHOOKE, (1.0, 10.0), u)
    y = (H @ x).reshape(-1, 3)
    nodes = np.array([0, 7, 40, mesh.n_nodes - 1])
    loc = d.apply_at_nodes(materials.NEOHOOKE, (1.0, 10.0), nodes, x, u)
    np.testing.assert_allclose(loc, y[nodes], atol=1e-12 * np.abs(y).max())
