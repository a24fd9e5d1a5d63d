"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds the only code both sides share: structured hexahedral box
meshes, Dirichlet DOF sets, initial conditions, material constants and the
per-element stiffness scale of the heterogeneous slab. It contains none of the
propagator's arithmetic (no shape-function gradients, quadrature, stresses,
mass, Krylov or exponential): only geometry, index bookkeeping and random
numbers.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds. Uniforms take the top 53 bits; normals use
the Box-Muller transform. The stream is portable (same bits on x86 and Arm).

Node numbering is lexicographic, ``n = i + NX*(j + NY*k)``; element local nodes
are lexicographic too, local index ``a + (p+1)*(b + (p+1)*c)`` for polynomial
order ``p`` and local lattice coordinates ``a, b, c`` in ``0..p``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First ``n`` outputs of SplitMix64 started from state ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``n`` doubles uniform on [lo, hi) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, n: int) -> np.ndarray:
    """``n`` standard normals by Box-Muller on pairs of SplitMix64 uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    out = np.empty(2 * m)
    out[0::2] = z[:m]
    out[1::2] = z[m:]
    return out[:n]


@dataclass
class BoxMesh:
    """A structured box of hexahedra (Q1: 8 nodes, Q2: 27 nodes per element)."""

    order: int
    nel: tuple  # elements per axis (nx, ny, nz)
    lengths: tuple  # box edge lengths (Lx, Ly, Lz)
    coords: np.ndarray  # (n_nodes, 3) float64
    conn: np.ndarray  # (n_elems, (order+1)^3) int32, lexicographic local order

    @property
    def n_nodes(self) -> int:
        return self.coords.shape[0]

    @property
    def n_elems(self) -> int:
        return self.conn.shape[0]

    @property
    def nodes_per_axis(self) -> tuple:
        return tuple(self.order * n + 1 for n in self.nel)


def box_mesh(order: int, nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float) -> BoxMesh:
    """Uniform box [0,Lx]x[0,Ly]x[0,Lz] split into nx*ny*nz hexahedra of order 1 or 2."""
    if order not in (1, 2):
        raise ValueError("order must be 1 or 2")
    NX, NY, NZ = order * nx + 1, order * ny + 1, order * nz + 1
    x = np.linspace(0.0, Lx, NX)
    y = np.linspace(0.0, Ly, NY)
    z = np.linspace(0.0, Lz, NZ)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    p1 = order + 1
    ek, ej, ei = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ei, ej, ek = ei.ravel(), ej.ravel(), ek.ravel()
    conn = np.empty((nx * ny * nz, p1 ** 3), dtype=np.int64)
    for c in range(p1):
        for b in range(p1):
            for a in range(p1):
                i = order * ei + a
                j = order * ej + b
                k = order * ek + c
                conn[:, a + p1 * (b + p1 * c)] = i + NX * (j + NY * k)
    return BoxMesh(order, (nx, ny, nz), (Lx, Ly, Lz), coords, conn.astype(np.int32))


def perturb_interior(mesh: BoxMesh, seed: int, frac: float = 0.15) -> BoxMesh:
    """Move interior nodes by up to ``frac`` of the node spacing (non-affine elements).

    For Q2 only vertex nodes move; edge, face and cell nodes are re-placed at the
    averages of their lattice neighbours so elements stay well shaped.
    """
    NX, NY, NZ = mesh.nodes_per_axis
    h = np.array(mesh.lengths) / (np.array([NX, NY, NZ]) - 1)
    c = mesh.coords.reshape(NZ, NY, NX, 3).copy()
    d = uniform(seed, c.size, -1.0, 1.0).reshape(c.shape) * frac * h
    p = mesh.order
    interior = np.zeros((NZ, NY, NX), dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    vert = np.zeros_like(interior)
    vert[::p, ::p, ::p] = True
    move = interior & vert
    c[move] += d[move]
    if p == 2:
        # mid-edge nodes along x, then y, then z, then face and cell centres
        c[:, :, 1::2] = 0.5 * (c[:, :, 0:-1:2] + c[:, :, 2::2])
        c[:, 1::2, :] = 0.5 * (c[:, 0:-1:2, :] + c[:, 2::2, :])
        c[1::2, :, :] = 0.5 * (c[0:-1:2, :, :] + c[2::2, :, :])
    return BoxMesh(mesh.order, mesh.nel, mesh.lengths, c.reshape(-1, 3), mesh.conn.copy())


def fixed_dofs_on_plane(mesh: BoxMesh, axis: int, value: float, comps=(0, 1, 2)) -> np.ndarray:
    """Global DOF indices (3*node + comp) of nodes on the plane x_axis == value."""
    nodes = np.nonzero(np.abs(mesh.coords[:, axis] - value) < 1e-12)[0]
    dofs = (3 * nodes[:, None] + np.array(comps)[None, :]).ravel()
    return np.sort(dofs).astype(np.int32)


# Euler-Bernoulli clamped-free first bending mode, beta*L = 1.8751 and
# sigma = 0.7341 (Blevins, "Formulas for natural frequency and mode shape",
# Table 8-1, clamped-free beam).
EB_BETA_L = 1.875104068711961
EB_SIGMA = 0.7340955137589


def eb_mode1(x: np.ndarray, L: float) -> np.ndarray:
    """Clamped-free first bending mode shape normalised to 1 at the free end."""
    def raw(s):
        b = EB_BETA_L * s
        return np.cosh(b) - np.cos(b) - EB_SIGMA * (np.sinh(b) - np.sin(b))
    return raw(np.asarray(x) / L) / raw(1.0)


def eb_omega1(E: float, rho: float, width: float, height: float, L: float) -> float:
    """First clamped-free bending frequency of a rectangular Euler-Bernoulli beam."""
    I = width * height ** 3 / 12.0
    A = width * height
    return EB_BETA_L ** 2 * math.sqrt(E * I / (rho * A * L ** 4))


MAT_LINEAR, MAT_NEOHOOKE, MAT_MOONEY_RIVLIN, MAT_SVK, MAT_YEOH = 0, 1, 2, 3, 4
MATERIAL_NAMES = {0: "linear", 1: "neohooke", 2: "mooney_rivlin", 3: "svk", 4: "yeoh"}


def lame_from_E_nu(E: float, nu: float):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def small_strain_moduli(kind: int, params) -> tuple:
    """(lambda, mu) of the material's response at zero strain (for dt and mode recipes)."""
    if kind == MAT_LINEAR:
        return lame_from_E_nu(*params[:2])
    if kind == MAT_NEOHOOKE:
        return params[1], params[0]
    if kind == MAT_MOONEY_RIVLIN:
        c10, c01, kappa = params[:3]
        mu = 2.0 * (c10 + c01)
        return kappa - 2.0 * mu / 3.0, mu
    if kind == MAT_SVK:
        return params[0], params[1]
    if kind == MAT_YEOH:
        c10, d1 = params[0], params[3]
        mu = 2.0 * c10
        return 2.0 / d1 - 2.0 * mu / 3.0, mu
    raise ValueError(kind)


@dataclass
class Problem:
    """One propagation workload: mesh, Dirichlet set, material, initial state, schedule."""

    name: str
    mesh: BoxMesh
    fixed_dofs: np.ndarray
    material: int
    params: tuple
    rho: float
    u0: np.ndarray  # (3*n_nodes,) float64, node-major (3*node + comp)
    v0: np.ndarray
    dt: float
    steps: int
    tol: float
    m_cap: int
    elem_scale: np.ndarray | None = None  # (n_elems,) float32 or None
    notes: dict = field(default_factory=dict)
    load: np.ndarray | None = None  # (3*n_nodes,) constant external nodal forces, or None

    @property
    def n_dofs(self) -> int:
        return 3 * self.mesh.n_nodes


def cfl_dt(mesh: BoxMesh, kind: int, params, rho: float, cfl: float) -> float:
    """dt = cfl * (smallest node spacing) / (dilatational wave speed at zero strain)."""
    lam, mu = small_strain_moduli(kind, params)
    cp = math.sqrt((lam + 2.0 * mu) / rho)
    NX, NY, NZ = mesh.nodes_per_axis
    h = min(L / (n - 1) for L, n in zip(mesh.lengths, (NX, NY, NZ)))
    return cfl * h / cp


def seed_of(k: int) -> int:
    return 20240508 + k


def beam_linear(nel=(20, 2, 2), seed=None) -> Problem:
    """Linear cantilever 10x1x1 (Q1), clamped at x=0, first-bending-mode velocity."""
    seed = seed_of(1) if seed is None else seed
    Lx, Ly, Lz = 10.0, 1.0, 1.0
    mesh = box_mesh(1, *nel, Lx, Ly, Lz)
    fixed = fixed_dofs_on_plane(mesh, 0, 0.0)
    amp = uniform(seed, 1, 0.01, 0.1)[0]
    u0 = np.zeros(3 * mesh.n_nodes)
    v0 = np.zeros(3 * mesh.n_nodes)
    v0[1::3] = amp * eb_mode1(mesh.coords[:, 0], Lx)
    v0[fixed] = 0.0
    return Problem("beam-linear-q1", mesh, fixed, MAT_LINEAR, (1.0e3, 0.3), 1.0, u0, v0,
                   dt=0.05, steps=200, tol=1e-10, m_cap=128, notes={"amplitude": amp})


def beam_linear_impulse(nel=(80, 8, 8), seed=None, width=0.3) -> Problem:
    """Linear cantilever 10x1x1 (Q1), clamped at x=0, struck near the tip: a transverse velocity
    patch exp(-r^2 / (2 width^2)) around (9.5, 0.5, 1.0) with a seeded amplitude in [0.01, 0.1]
    (broadband: many modes carry energy, as under the paper's impulsive loads)."""
    seed = seed_of(1) if seed is None else seed
    Lx, Ly, Lz = 10.0, 1.0, 1.0
    mesh = box_mesh(1, *nel, Lx, Ly, Lz)
    fixed = fixed_dofs_on_plane(mesh, 0, 0.0)
    amp = uniform(seed, 1, 0.01, 0.1)[0]
    r2 = ((mesh.coords - np.array([9.5, 0.5, 1.0])) ** 2).sum(axis=1)
    u0 = np.zeros(3 * mesh.n_nodes)
    v0 = np.zeros(3 * mesh.n_nodes)
    v0[1::3] = amp * np.exp(-r2 / (2 * width ** 2))
    v0[fixed] = 0.0
    return Problem("beam-linear-impulse-q1", mesh, fixed, MAT_LINEAR, (1.0e3, 0.3), 1.0, u0, v0,
                   dt=0.05, steps=20, tol=1e-8, m_cap=128, notes={"amplitude": amp, "width": width})


def beam_neohooke(nel=(80, 8, 8), dt=0.02, seed=None, steps=500, jitter=True, amp_scale=1.0) -> Problem:
    """Neo-Hookean cantilever 20x2x2 (Q1), clamped at x=0, ~10% tip deflection."""
    seed = seed_of(2) if seed is None else seed
    Lx, Ly, Lz = 20.0, 2.0, 2.0
    mu, lam = 345.0, 805.0
    mesh = box_mesh(1, *nel, Lx, Ly, Lz)
    fixed = fixed_dofs_on_plane(mesh, 0, 0.0)
    E = mu * (3 * lam + 2 * mu) / (lam + mu)
    w1 = eb_omega1(E, 1.0, Lz, Ly, Lx)
    amp = amp_scale * 0.1 * Lx * w1  # linearised mode-1 velocity for a tip deflection of 0.1*Lx
    jitter = 0.9 + 0.2 * uniform(seed, mesh.n_nodes) if jitter else 1.0
    u0 = np.zeros(3 * mesh.n_nodes)
    v0 = np.zeros(3 * mesh.n_nodes)
    v0[1::3] = amp * eb_mode1(mesh.coords[:, 0], Lx) * jitter
    v0[fixed] = 0.0
    return Problem("beam-neohooke-q1", mesh, fixed, MAT_NEOHOOKE, (mu, lam), 1.0, u0, v0,
                   dt=dt, steps=steps, tol=1e-8, m_cap=128, notes={"amplitude": amp, "omega1": w1})


def rubber_block(n=32, seed=None, steps=200, cfl=6.0) -> Problem:
    """Neo-Hookean unit cube (Q2), bottom face fixed, compressive top-down velocity."""
    seed = seed_of(3) if seed is None else seed
    mu, lam = 1.0, 10.0
    mesh = box_mesh(2, n, n, n, 1.0, 1.0, 1.0)
    fixed = fixed_dofs_on_plane(mesh, 2, 0.0)
    c = uniform(seed, 4, -0.1, 0.1)
    x, y, z = mesh.coords[:, 0], mesh.coords[:, 1], mesh.coords[:, 2]
    g = np.ones_like(x)
    idx = 0
    for kk in (1, 2):
        for ll in (1, 2):
            g += c[idx] * np.cos(kk * np.pi * x) * np.cos(ll * np.pi * y)
            idx += 1
    u0 = np.zeros(3 * mesh.n_nodes)
    v0 = np.zeros(3 * mesh.n_nodes)
    v0[2::3] = -0.1 * z * g
    v0[fixed] = 0.0
    dt = cfl_dt(mesh, MAT_NEOHOOKE, (mu, lam), 1.0, cfl)
    return Problem("rubber-neohooke-q2", mesh, fixed, MAT_NEOHOOKE, (mu, lam), 1.0, u0, v0,
                   dt=dt, steps=steps, tol=1e-8, m_cap=64, notes={"c_kl": c.tolist(), "cfl": cfl})


def tissue_slab(nel=(256, 128, 128), seed=None, steps=50, cfl=6.0) -> Problem:
    """Mooney-Rivlin 2x1x1 slab (Q1), x=0 fixed, lognormal stiffness, velocity patch at x=2."""
    seed = seed_of(4) if seed is None else seed
    c10, c01 = 0.5, 0.05
    kappa = 1.0e3 * 2.0 * (c10 + c01)
    mesh = box_mesh(1, *nel, 2.0, 1.0, 1.0)
    fixed = fixed_dofs_on_plane(mesh, 0, 0.0)
    scale = np.exp(0.1 * normal(seed, mesh.n_elems)).astype(np.float32)
    r2 = ((mesh.coords - np.array([2.0, 0.5, 0.5])) ** 2).sum(axis=1)
    u0 = np.zeros(3 * mesh.n_nodes)
    v0 = np.zeros(3 * mesh.n_nodes)
    v0[0::3] = -0.05 * np.exp(-r2 / (2 * 0.1 ** 2))
    v0[fixed] = 0.0
    dt = cfl_dt(mesh, MAT_MOONEY_RIVLIN, (c10, c01, kappa), 1.0, cfl)
    return Problem("tissue-mooney-rivlin-q1", mesh, fixed, MAT_MOONEY_RIVLIN, (c10, c01, kappa), 1.0,
                   u0, v0, dt=dt, steps=steps, tol=1e-6, m_cap=64, elem_scale=scale,
                   notes={"cfl": cfl})


def with_face_load(prob: Problem, total: float, comp: int = 1, axis: int = 0) -> Problem:
    """Copy of `prob` with a constant traction on the face x_axis = max: `total` force in
    direction `comp`, split equally over that face's free nodes (the paper's P != 0 case)."""
    import dataclasses
    x = prob.mesh.coords[:, axis]
    face = np.flatnonzero(np.isclose(x, x.max()))
    fixed = set(int(d) for d in prob.fixed_dofs)
    nodes = [n for n in face if 3 * int(n) + comp not in fixed]
    P = np.zeros(3 * prob.mesh.n_nodes)
    P[3 * np.asarray(nodes, dtype=np.int64) + comp] = total / len(nodes)
    return dataclasses.replace(prob, load=P, notes=dict(prob.notes, load_total=total))


def make_problem(name: str, **kw) -> Problem:
    table = {
        "beam-linear-q1": beam_linear,
        "beam-neohooke-q1": beam_neohooke,
        "rubber-neohooke-q2": rubber_block,
        "tissue-mooney-rivlin-q1": tissue_slab,
    }
    return table[name](**kw)


def served_mix(n_requests=256, seed=None, rate_hz=50.0, dof_range=(2000, 500000),
               horizon=(50, 1000), horizon_scale=1.0):
    """The served mixed batch: Poisson arrivals of Q1 beams (10:1:1) and blocks (1:1:1).

    Each request draws: shape (beam or block), DOFs log-uniform in dof_range
    (nearest structured box), material linear or Neo-Hookean (50/50) with mu
    log-uniform in [1, 10] and lambda/mu log-uniform in [1, 10], rho = 1,
    dt = c / omega_max with c log-uniform in [4, 32] and
    omega_max = 2 sqrt(3) c_p / h, a horizon uniform in `horizon` steps (times
    horizon_scale), tol 1e-8. Returns a list of (arrival_s, Problem, steps).
    """
    seed = seed_of(5) if seed is None else seed
    u = uniform(seed, 16 * n_requests).reshape(n_requests, 16)
    arrivals = np.cumsum(-np.log(1.0 - u[:, 0]) / rate_hz)
    out = []
    for k in range(n_requests):
        beam = u[k, 1] < 0.5
        n_dof = math.exp(math.log(dof_range[0]) + u[k, 2] * math.log(dof_range[1] / dof_range[0]))
        nonlinear = u[k, 3] < 0.5
        mu = 10.0 ** u[k, 4]
        lam = mu * 10.0 ** u[k, 5]
        c = math.exp(math.log(4.0) + u[k, 6] * math.log(8.0))
        steps = int(round(horizon[0] + u[k, 7] * (horizon[1] - horizon[0])))
        steps = max(1, int(round(steps * horizon_scale)))
        if beam:
            m_ = max(1, int(round((n_dof / 30.0) ** (1.0 / 3.0))))
            nel, L = (10 * m_, m_, m_), (10.0, 1.0, 1.0)
        else:
            m_ = max(1, int(round((n_dof / 3.0) ** (1.0 / 3.0))) - 1)
            nel, L = (m_, m_, m_), (1.0, 1.0, 1.0)
        mesh = box_mesh(1, *nel, *L)
        if beam:
            fixed = fixed_dofs_on_plane(mesh, 0, 0.0)
        else:
            fixed = fixed_dofs_on_plane(mesh, 2, 0.0)
        if nonlinear:
            kind, params = MAT_NEOHOOKE, (mu, lam)
        else:
            kind, params = MAT_LINEAR, (mu * (3 * lam + 2 * mu) / (lam + mu), lam / (2 * (lam + mu)))
        cp = math.sqrt(lam + 2 * mu)
        h = min(Li / n for Li, n in zip(L, nel))
        dt = c / (2.0 * math.sqrt(3.0) * cp / h)
        u0 = np.zeros(3 * mesh.n_nodes)
        v0 = np.zeros(3 * mesh.n_nodes)
        if beam:
            E = mu * (3 * lam + 2 * mu) / (lam + mu)
            v0[1::3] = 0.01 * L[0] * eb_omega1(E, 1.0, L[2], L[1], L[0]) * eb_mode1(mesh.coords[:, 0], L[0])
        else:
            v0[2::3] = -0.01 * cp * mesh.coords[:, 2]
        v0[fixed] = 0.0
        prob = Problem(f"served-{k}", mesh, fixed, kind, params, 1.0, u0, v0, dt=dt, steps=steps,
                       tol=1e-8, m_cap=64, notes={"beam": bool(beam), "c": c})
        out.append((float(arrivals[k]), prob, steps))
    return out
