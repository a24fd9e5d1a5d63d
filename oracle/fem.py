"""FP64 finite-element discretisation for the oracle (test infrastructure only).

This package is the plain, slow reference the CUDA path is checked against. Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it; the product path never does.

What this file computes, by passage of the paper (arXiv 2405.05213):

* Section 2.2, Eq. "expansion in finite-element basis": hexahedral Lagrange
  elements (here order 1 or 2), interpolated isoparametrically.
* Section 2.2, Eq. "weak form term 2": the internal force
  ``R_A = sum_e int_e B_A^T S dV``, written with the first Piola stress
  ``P = F S`` as ``R_{A,i} = int P_iJ dN_A/dX_J dV`` (the same contraction).
* Section 2.2, closing paragraph: Gauss quadrature for the stiffness terms,
  Gauss-Lobatto-Legendre (GLL) quadrature for the mass, which makes the mass
  matrix diagonal.
* Section 2.3, Eq. "discrete dynamic equilibrium using H": the H-matrix is
  assembled from the secant stress ``P_lin(G; u*)`` of ``oracle.materials``,
  so that ``H(u*) x = sum_e int P_lin(grad x; grad u*) : grad N dV``.

Dirichlet DOFs are eliminated (rows and columns removed); the state at those
DOFs is identically zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import materials


# ---------------------------------------------------------------- 1D bases
def lagrange_nodes(order: int) -> np.ndarray:
    """Equispaced Lagrange nodes on [-1, 1] (they are also the GLL points for p = 1, 2)."""
    return np.linspace(-1.0, 1.0, order + 1)


def lagrange_1d(order: int, xi: np.ndarray):
    """Values and derivatives of the 1D Lagrange basis at points ``xi``.

    Returns ``(N, dN)`` with shapes ``(len(xi), order+1)``; built from the
    product formula ``N_a(x) = prod_{b != a} (x - x_b) / (x_a - x_b)``.
    """
    xn = lagrange_nodes(order)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    n = order + 1
    N = np.ones((xi.size, n))
    dN = np.zeros((xi.size, n))
    for a in range(n):
        others = [b for b in range(n) if b != a]
        for b in others:
            N[:, a] *= (xi - xn[b]) / (xn[a] - xn[b])
        for c in others:  # derivative of the product: sum over the dropped factor
            term = np.full(xi.size, 1.0 / (xn[a] - xn[c]))
            for b in others:
                if b != c:
                    term *= (xi - xn[b]) / (xn[a] - xn[b])
            dN[:, a] += term
    return N, dN


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (numpy's library routine)."""
    return np.polynomial.legendre.leggauss(n)


def gll(n: int):
    """n-point Gauss-Lobatto-Legendre rule on [-1, 1] for n = 2, 3."""
    if n == 2:
        return np.array([-1.0, 1.0]), np.array([1.0, 1.0])
    if n == 3:
        return np.array([-1.0, 0.0, 1.0]), np.array([1.0, 4.0, 1.0]) / 3.0
    raise ValueError("GLL rule implemented for n = 2, 3 only")


# ---------------------------------------------------------------- 3D tensor products
def shape_3d(order: int, pts1d: np.ndarray, w1d: np.ndarray):
    """Tensor-product shape functions at the tensor grid of ``pts1d``.

    Returns ``N (nq, nen)``, ``dN (nq, nen, 3)`` (derivatives in the reference
    coordinates xi, eta, zeta) and weights ``w (nq,)``. Quadrature points and
    local nodes are both ordered lexicographically with the first index fastest.
    """
    N1, dN1 = lagrange_1d(order, pts1d)
    nq1, n1 = N1.shape
    nq, nen = nq1 ** 3, n1 ** 3
    N = np.empty((nq, nen))
    dN = np.empty((nq, nen, 3))
    w = np.empty(nq)
    for qz in range(nq1):
        for qy in range(nq1):
            for qx in range(nq1):
                q = qx + nq1 * (qy + nq1 * qz)
                w[q] = w1d[qx] * w1d[qy] * w1d[qz]
                for c in range(n1):
                    for b in range(n1):
                        for a in range(n1):
                            A = a + n1 * (b + n1 * c)
                            N[q, A] = N1[qx, a] * N1[qy, b] * N1[qz, c]
                            dN[q, A, 0] = dN1[qx, a] * N1[qy, b] * N1[qz, c]
                            dN[q, A, 1] = N1[qx, a] * dN1[qy, b] * N1[qz, c]
                            dN[q, A, 2] = N1[qx, a] * N1[qy, b] * dN1[qz, c]
    return N, dN, w


class Discretisation:
    """Mesh-dependent FE data: quadrature, gradients, mass, free-DOF numbering.

    ``coords (n_nodes, 3)``, ``conn (n_elems, nen)`` lexicographic local order,
    ``fixed_dofs`` global DOF ids ``3*node + comp`` with zero displacement.
    """

    def __init__(self, order, coords, conn, fixed_dofs, rho=1.0, elem_scale=None):
        self.order = int(order)
        self.coords = np.asarray(coords, dtype=np.float64)
        self.conn = np.asarray(conn, dtype=np.int64)
        self.n_nodes = self.coords.shape[0]
        self.n_elems, self.nen = self.conn.shape
        assert self.nen == (self.order + 1) ** 3
        self.N = 3 * self.n_nodes
        self.rho = float(rho)
        self.elem_scale = (np.ones(self.n_elems) if elem_scale is None
                           else np.asarray(elem_scale, dtype=np.float64))
        # Gauss-Legendre with order+1 points per axis (full integration)
        gp, gw = gauss_legendre(self.order + 1)
        self.Nq, self.dNref, self.wq = shape_3d(self.order, gp, gw)
        self._geo = None  # element geometry at the Gauss points, built on first use
        # free DOF numbering (Dirichlet elimination)
        fixed = np.zeros(self.N, dtype=bool)
        fixed[np.asarray(fixed_dofs, dtype=np.int64)] = True
        self.fixed = fixed
        self.free = np.nonzero(~fixed)[0]
        self.Nf = self.free.size
        self.mass = self._gll_mass()  # per global DOF (3 equal entries per node)
        self.mf = self.mass[self.free]

    # -- geometry -------------------------------------------------------
    @property
    def gradN(self):
        if self._geo is None:
            self._geo = self._geometry(self.dNref, self.wq)
        return self._geo[0]

    @property
    def dV(self):
        if self._geo is None:
            self._geo = self._geometry(self.dNref, self.wq)
        return self._geo[1]

    def _geometry(self, dNref, wq, elems=None):
        """Physical gradients dN/dX (ne, nq, nen, 3) and dV = w*detJ (ne, nq)."""
        conn = self.conn if elems is None else self.conn[elems]
        X = self.coords[conn]  # (ne, nen, 3)
        # J_{iJ} = dX_i / dxi_J
        J = np.einsum("eai,qaj->eqij", X, dNref)
        detJ = np.linalg.det(J)
        if np.any(detJ <= 0):
            raise ValueError("inverted element in the reference configuration")
        Jinv = np.linalg.inv(J)
        # dN/dX_i = sum_J dN/dxi_J (J^-1)_{J i}
        gradN = np.einsum("qaj,eqji->eqai", dNref, Jinv)
        return gradN, detJ * wq[None, :]

    def _gll_mass(self):
        """Diagonal mass by GLL nodal quadrature (Section 2.2): M_A = sum_e rho w_A detJ(xi_A)."""
        pts, w1 = gll(self.order + 1)
        _, dN_at_nodes, w = shape_3d(self.order, pts, w1)
        X = self.coords[self.conn]
        J = np.einsum("eai,qaj->eqij", X, dN_at_nodes)
        detJ = np.linalg.det(J)
        # GLL points coincide with the element nodes: point q is local node q
        contrib = self.rho * detJ * w[None, :]  # (ne, nen)
        m_node = np.zeros(self.n_nodes)
        np.add.at(m_node, self.conn.ravel(), contrib.ravel())
        return np.repeat(m_node, 3)

    # -- fields -----------------------------------------------------------
    def grad(self, u_full, gradN=None, conn=None):
        """Displacement gradient D_{iJ} = sum_A u_{A,i} dN_A/dX_J at all Gauss points."""
        gradN = self.gradN if gradN is None else gradN
        conn = self.conn if conn is None else conn
        ue = u_full.reshape(-1, 3)[conn]  # (ne, nen, 3)
        return np.einsum("eai,eqaj->eqij", ue, gradN)

    def to_full(self, x_free):
        out = np.zeros(self.N)
        out[self.free] = x_free
        return out

    # -- internal force and energy ---------------------------------------
    def internal_force(self, kind, params, u_full):
        """R(u) of Eq. "weak form term 2", full length 3*n_nodes."""
        D = self.grad(u_full)
        P = materials.pk1(kind, params, np.eye(3) + D)
        P = P * self.elem_scale[:, None, None, None]
        fe = np.einsum("eqij,eqaj,eq->eai", P, self.gradN, self.dV)
        R = np.zeros((self.n_nodes, 3))
        np.add.at(R, self.conn.ravel(), fe.reshape(-1, 3))
        return R.ravel()

    def strain_energy(self, kind, params, u_full):
        """sum_e sum_q psi(F) w detJ: the stored energy with the stiffness quadrature."""
        D = self.grad(u_full)
        psi = materials.psi(kind, params, np.eye(3) + D)
        return float(np.sum(psi * self.dV * self.elem_scale[:, None]))

    # -- H-matrix assembly -------------------------------------------------
    def element_matrices(self, kind, params, ustar_full, elems=None, tangent=False):
        """Element blocks of H(u*) (ne, nen*3, nen*3), DOF order 3*A + i.

        ``P_lin`` is linear in G, so its action on the nine unit tensors
        e_k (x) e_L gives the 9x9 operator T with
        ``P_lin(G)_iJ = T[iJ, kL] G_kL``; then
        ``H_e[Ai, Bk] = sum_q dV_q dN_A/dX_J T[iJ, kL] dN_B/dX_L``.
        With ``tangent=True`` T is instead dP/dF at F = I + grad u* (the
        consistent tangent, by central differences of P), giving dR/du.
        """
        if elems is None:
            gradN, dV, conn, scale = self.gradN, self.dV, self.conn, self.elem_scale
        else:
            gradN, dV = self._geometry(self.dNref, self.wq, elems)
            conn, scale = self.conn[elems], self.elem_scale[elems]
        Dstar = None
        if ustar_full is not None:
            Dstar = self.grad(ustar_full, gradN, conn)
        ne, nq = dV.shape
        T = np.empty((ne, nq, 3, 3, 3, 3))
        F0 = np.eye(3) + (np.zeros((ne, nq, 3, 3)) if Dstar is None else Dstar)
        for k in range(3):
            for L in range(3):
                G = np.zeros((ne, nq, 3, 3))
                G[..., k, L] = 1.0
                if tangent:
                    h = 1e-6
                    T[..., k, L] = (materials.pk1(kind, params, F0 + h * G)
                                    - materials.pk1(kind, params, F0 - h * G)) / (2 * h)
                else:
                    T[..., k, L] = materials.plin(kind, params, G, Dstar)
        W = np.einsum("eqaj,eqijkl->eqaikl", gradN, T * (dV * scale[:, None])[:, :, None, None, None, None],
                      optimize=True)
        He = np.einsum("eqaikl,eqbl->eaibk", W, gradN, optimize=True)
        nen = conn.shape[1]
        return He.reshape(ne, 3 * nen, 3 * nen)

    def assemble_H(self, kind, params, ustar_full, chunk=4096, tangent=False):
        """Assembled H(u*) (or the tangent dR/du) restricted to the free DOFs, scipy CSR (FP64)."""
        rows, cols, vals = [], [], []
        nen = self.nen
        for e0 in range(0, self.n_elems, chunk):
            elems = np.arange(e0, min(e0 + chunk, self.n_elems))
            He = self.element_matrices(kind, params, ustar_full, elems, tangent)
            dofs = (3 * self.conn[elems][:, :, None] + np.arange(3)[None, None, :]).reshape(len(elems), 3 * nen)
            rows.append(np.repeat(dofs, 3 * nen, axis=1).ravel())
            cols.append(np.tile(dofs, (1, 3 * nen)).ravel())
            vals.append(He.ravel())
        rows = np.concatenate(rows)
        cols = np.concatenate(cols)
        vals = np.concatenate(vals)
        H = sp.csr_matrix((vals, (rows, cols)), shape=(self.N, self.N))
        return H[self.free][:, self.free].tocsr()

    def scaled(self, H):
        """H-bar = M^{-1/2} H M^{-1/2} on the free DOFs (Section 2.3)."""
        s = 1.0 / np.sqrt(self.mf)
        return sp.diags(s) @ H @ sp.diags(s)

    # -- local apply at selected nodes (for sampled checks at large sizes) --
    def apply_at_nodes(self, kind, params, nodes, x_full, ustar_full=None):
        """(H(u*) x) at the given nodes only, by summing their incident elements.

        Returns an array (len(nodes), 3). Fixed DOFs are not masked here.
        """
        nodes = np.asarray(nodes, dtype=np.int64)
        hit = np.isin(self.conn, nodes).any(axis=1)
        elems = np.nonzero(hit)[0]
        He = self.element_matrices(kind, params, ustar_full, elems)
        xe = x_full.reshape(-1, 3)[self.conn[elems]].reshape(len(elems), -1)
        ye = np.einsum("eab,eb->ea", He, xe).reshape(len(elems), self.nen, 3)
        pos = {int(n): i for i, n in enumerate(nodes)}
        out = np.zeros((len(nodes), 3))
        for e_local, e in enumerate(elems):
            for A, n in enumerate(self.conn[e]):
                i = pos.get(int(n))
                if i is not None:
                    out[i] += ye[e_local, A]
        return out
