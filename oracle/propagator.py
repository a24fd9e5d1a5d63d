"""The exponential propagator time step, FP64 (test infrastructure).

Passages of arXiv 2405.05213 followed:

* Section 2.3: mass scaling ``u_bar = M^{1/2} u``, ``H_bar = M^{-1/2} H M^{-1/2}``
  and the first-order recast ``d/dt w_bar = A w_bar`` with
  ``A = [[0, I], [-H_bar(u), 0]]`` (Eq. "A expression at P=0"). With a constant
  external load P the state is augmented by a last entry 1 and A gains the
  column ``P_bar = M^{-1/2} P`` in the velocity rows
  (Eq. "A expression at P != 0"): ``A = [[0, I, 0], [-H_bar, 0, P_bar], [0, 0, 0]]``.
* Section 3, Eqs. "MagnusEquation", "compositionProperty", "temporalDisc",
  "truncOmegaB": one step applies the first Magnus term ``exp(Omega)``.
* Section 4.1, Eq. "quadratureApprox": midpoint rule,
  ``Omega ~= dt A(t_{n-1} + dt/2)``.
* Section 4.2: predictor-corrector for the midpoint operator. The predictor
  operator is the linear extrapolation of H_bar from the two previous
  midpoints to ``t_{n-1} + dt/4``: ``1.75 H_bar(u_{n-3/2}) - 0.75 H_bar(u_{n-5/2})``
  (constant extrapolation while fewer than two midpoints exist: step 1 uses
  ``H_bar(u_0)``, step 2 uses ``H_bar(u_{1/2})``). It propagates ``w_bar_{n-1}``
  by dt/2; ``H_bar(u_{n-1/2})`` is then built once and propagates
  ``w_bar_{n-1}`` by the full dt.
* Section 4.3: ``exp(tau A) w`` by Arnoldi (``oracle.krylov``).
* Section 5.2, Eq. "energyExpr": ``E = v_bar^T v_bar / 2 + u_bar^T H_bar u_bar / 2``
  (linear); for nonlinear materials the potential part is the stored energy
  ``sum_e sum_q psi(F) w detJ`` with the stiffness quadrature. With a constant
  load the potential of the load, ``-P^T u = -P_bar^T u_bar``, is added (the
  conserved total energy of a conservative load).

Linear material: ``H(u) = K`` and one Krylov solve per step.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import materials
from .fem import Discretisation
from .krylov import arnoldi_expv


@dataclass
class StepLog:
    m: list = field(default_factory=list)
    eps: list = field(default_factory=list)
    converged: list = field(default_factory=list)


class Propagator:
    """State ``w_bar = [M^{1/2} u; M^{1/2} v]`` on the free DOFs and its time steps."""

    def __init__(self, order, coords, conn, fixed_dofs, kind, params, rho, u0, v0,
                 elem_scale=None, m_cap=128, load=None):
        self.fe = Discretisation(order, coords, conn, fixed_dofs, rho, elem_scale)
        self.kind = int(kind)
        self.params = tuple(float(p) for p in params)
        self.m_cap = int(m_cap)
        fe = self.fe
        self.sqm = np.sqrt(fe.mf)
        u0 = np.asarray(u0, dtype=np.float64)
        v0 = np.asarray(v0, dtype=np.float64)
        self.w = np.concatenate([self.sqm * u0[fe.free], self.sqm * v0[fe.free]])
        self.pbar = None  # P_bar on the free DOFs (constant load), or None
        if load is not None:
            P = np.asarray(load, dtype=np.float64)
            self.pbar = P[fe.free] / self.sqm
            self.w = np.concatenate([self.w, [1.0]])  # augmented state [u_bar; v_bar; 1]
        self.t_index = 0
        self.mid_history = []  # physical midpoint displacements u_{k-1/2}, newest last
        self.log = StepLog()
        self._Hbar_lin = None

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(prob.mesh.order, prob.mesh.coords, prob.mesh.conn, prob.fixed_dofs,
                   prob.material, prob.params, prob.rho, prob.u0, prob.v0,
                   elem_scale=prob.elem_scale, m_cap=kw.pop("m_cap", prob.m_cap),
                   load=kw.pop("load", getattr(prob, "load", None)), **kw)

    # -- operators ----------------------------------------------------------
    @property
    def Nf(self):
        return self.fe.Nf

    def u_full(self, w=None):
        w = self.w if w is None else w
        return self.fe.to_full(w[: self.Nf] / self.sqm)

    def v_full(self, w=None):
        w = self.w if w is None else w
        return self.fe.to_full(w[self.Nf:2 * self.Nf] / self.sqm)

    def Hbar(self, ustar_full):
        """H_bar(u*) on the free DOFs (CSR)."""
        if self.kind == materials.LINEAR:
            if self._Hbar_lin is None:
                self._Hbar_lin = self.fe.scaled(self.fe.assemble_H(self.kind, self.params, None))
            return self._Hbar_lin
        return self.fe.scaled(self.fe.assemble_H(self.kind, self.params, ustar_full))

    def A_apply(self, Hbar):
        Nf = self.Nf
        if self.pbar is None:
            def apply(x):
                return np.concatenate([x[Nf:], -(Hbar @ x[:Nf])])
            return apply
        pbar = self.pbar

        def apply_aug(x):  # x = [u_bar; v_bar; xi]
            return np.concatenate([x[Nf:2 * Nf], -(Hbar @ x[:Nf]) + x[2 * Nf] * pbar, [0.0]])
        return apply_aug

    def expv(self, Hbar, tau, w, tol, m_fixed=0):
        return arnoldi_expv(self.A_apply(Hbar), w, tau, tol, self.m_cap, m_fixed)

    # -- time step ------------------------------------------------------------
    def step(self, dt, tol, m_fixed=0, m_fixed_pred=None):
        """One time step; returns (m, eps) of the last Krylov solve (the corrector)."""
        if self.kind == materials.LINEAR:
            r = self.expv(self.Hbar(None), dt, self.w, tol, m_fixed)
            self._record(r)
            self.w = r.w
            self.t_index += 1
            return r.m, r.eps
        hist = self.mid_history
        if len(hist) == 0:
            Hp = self.Hbar(self.u_full())
        elif len(hist) == 1:
            Hp = self.Hbar(hist[-1])
        else:
            Hp = 1.75 * self.Hbar(hist[-1]) - 0.75 * self.Hbar(hist[-2])
        mp = m_fixed if m_fixed_pred is None else m_fixed_pred
        rp = self.expv(Hp, 0.5 * dt, self.w, tol, mp)
        self._record(rp)
        u_half = self.u_full(rp.w)
        rc = self.expv(self.Hbar(u_half), dt, self.w, tol, m_fixed)
        self._record(rc)
        self.w = rc.w
        hist.append(u_half)
        if len(hist) > 2:
            hist.pop(0)
        self.t_index += 1
        return rc.m, rc.eps

    def _record(self, r):
        self.log.m.append(r.m)
        self.log.eps.append(r.eps)
        self.log.converged.append(r.converged)

    # -- energy -----------------------------------------------------------
    def energy(self):
        """(total, kinetic, potential)."""
        Nf = self.Nf
        ub, vb = self.w[:Nf], self.w[Nf:2 * Nf]
        ke = 0.5 * float(vb @ vb)
        if self.kind == materials.LINEAR:
            pe = 0.5 * float(ub @ (self.Hbar(None) @ ub))
        else:
            pe = self.fe.strain_energy(self.kind, self.params, self.u_full())
        if self.pbar is not None:
            pe -= float(self.pbar @ ub)
        return ke + pe, ke, pe


def run(prob, steps=None, dt=None, tol=None, m_fixed=0, m_cap=None):
    """Propagate a ``inputs.Problem`` and return the final Propagator."""
    kw = {} if m_cap is None else {"m_cap": m_cap}
    P = Propagator.from_problem(prob, **kw)
    steps = prob.steps if steps is None else steps
    dt = prob.dt if dt is None else dt
    tol = prob.tol if tol is None else tol
    for _ in range(steps):
        P.step(dt, tol, m_fixed)
    return P
