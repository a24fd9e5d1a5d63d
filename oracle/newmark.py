"""Newmark-beta (beta = 1/4, gamma = 1/2), the paper's comparison integrator, FP64.

Test infrastructure. Section 6 of arXiv 2405.05213 compares the exponential
propagator with the average-acceleration Newmark method (Newmark 1959). Here:

* linear: ``(M + beta dt^2 K) a_{n+1} = -K u_pred`` solved by a sparse direct
  factorisation (a library routine);
* nonlinear ("fully implicit"): Newton iterations on ``M a + R(u) = 0`` with
  the consistent tangent dR/du (``Discretisation.assemble_H(tangent=True)``)
  and a sparse direct solve per iteration.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import materials
from .fem import Discretisation


class Newmark:
    def __init__(self, order, coords, conn, fixed_dofs, kind, params, rho, u0, v0, elem_scale=None,
                 beta=0.25, gamma=0.5):
        self.fe = Discretisation(order, coords, conn, fixed_dofs, rho, elem_scale)
        self.kind, self.params = int(kind), tuple(params)
        self.beta, self.gamma = beta, gamma
        fe = self.fe
        self.u = np.asarray(u0, dtype=np.float64)[fe.free].copy()
        self.v = np.asarray(v0, dtype=np.float64)[fe.free].copy()
        self.a = -self._force(self.u) / fe.mf
        self._lu = None

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(prob.mesh.order, prob.mesh.coords, prob.mesh.conn, prob.fixed_dofs,
                   prob.material, prob.params, prob.rho, prob.u0, prob.v0, prob.elem_scale, **kw)

    def _force(self, u_free):
        fe = self.fe
        return fe.internal_force(self.kind, self.params, fe.to_full(u_free))[fe.free]

    def step(self, dt):
        b, g, fe = self.beta, self.gamma, self.fe
        u_pred = self.u + dt * self.v + dt * dt * (0.5 - b) * self.a
        v_pred = self.v + (1 - g) * dt * self.a
        if self.kind == materials.LINEAR:
            if self._lu is None or self._lu[0] != dt:
                K = fe.assemble_H(self.kind, self.params, None)
                S = (sp.diags(fe.mf) + b * dt * dt * K).tocsc()
                self._lu = (dt, spla.splu(S), K)
            _, lu, K = self._lu
            a_new = lu.solve(-(K @ u_pred))
        else:
            a_new = self.a.copy()
            for _ in range(30):
                u_new = u_pred + b * dt * dt * a_new
                res = fe.mf * a_new + self._force(u_new)
                if np.linalg.norm(res) <= 1e-12 * max(1.0, np.linalg.norm(fe.mf * a_new)):
                    break
                KT = fe.assemble_H(self.kind, self.params, fe.to_full(u_new), tangent=True)
                S = (sp.diags(fe.mf) + b * dt * dt * KT).tocsc()
                a_new = a_new + spla.spsolve(S, -res)
        self.u = u_pred + b * dt * dt * a_new
        self.v = v_pred + g * dt * a_new
        self.a = a_new

    def energy(self):
        ke = 0.5 * float(self.v @ (self.fe.mf * self.v))
        pe = self.fe.strain_energy(self.kind, self.params, self.fe.to_full(self.u))
        return ke + pe, ke, pe
