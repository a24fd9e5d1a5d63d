"""ctypes binding of libetp (include/etp.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts numpy
arrays (host) and torch tensors (device) to pointers and checks status codes.
There is no CPU fallback: if ``libetp.so`` is missing or cannot load, every
call raises.

The ``etp_*`` functions carry the C names and signatures; ``Context``,
``Mesh`` and ``Trajectory`` own the handles and release them.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libetp.so")

ETP_OK, ETP_ERR_INVALID, ETP_ERR_OOM, ETP_ERR_CUDA = 0, 1, 2, 3
ETP_ERR_NOT_CONVERGED, ETP_ERR_NONFINITE, ETP_ERR_INVERTED_ELEMENT = 4, 5, 6
ETP_ERR_TIMEOUT, ETP_ERR_IO = 7, 8
ETP_PREC_FP64, ETP_PREC_MIXED = 0, 1
ETP_MAT_LINEAR, ETP_MAT_NEOHOOKE, ETP_MAT_MOONEY_RIVLIN, ETP_MAT_SVK, ETP_MAT_YEOH = range(5)
ETP_KRYLOV_ARNOLDI, ETP_KRYLOV_LANCZOS_ENERGY = 0, 1
ETP_NUM_KERNEL_CLASSES = 11
KERNEL_CLASSES = ["elem_apply", "node_gather", "cgs_dot", "cgs_update_dot", "cgs_update_norm",
                  "small_expm", "state_combine", "other", "fused_arnoldi_step", "frozen_build", "lanczos"]


class EtpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libetp status {status}: {msg}")
        self.status = status


class StepInfo(C.Structure):
    _fields_ = [("m_pred", C.c_int), ("m_corr", C.c_int), ("eps_pred", C.c_double),
                ("eps_corr", C.c_double), ("beta", C.c_double), ("converged", C.c_int)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_F32 = C.POINTER(C.c_float)

_SIGS = {
    "etp_last_error": (C.c_char_p, []),
    "etp_version": (C.c_char_p, []),
    "etp_debug_spin_limit": (C.c_int, [_P, C.c_uint64]),
    "etp_ctx_create": (C.c_int, [C.c_int, _P, C.POINTER(_P)]),
    "etp_ctx_destroy": (None, [_P]),
    "etp_mesh_create": (C.c_int, [_P, C.c_int, C.c_int64, _D, C.c_int64, _I32, C.c_int64, _I32, C.POINTER(_P)]),
    "etp_mesh_destroy": (None, [_P]),
    "etp_material_set": (C.c_int, [_P, C.c_int, _D, C.c_int, C.c_double, _F32]),
    "etp_state_init": (C.c_int, [_P, _D, _D, C.c_int, C.c_int, C.c_int, C.POINTER(_P)]),
    "etp_traj_destroy": (None, [_P]),
    "etp_step": (C.c_int, [_P, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int), _D]),
    "etp_step_ex": (C.c_int, [_P, C.c_double, C.c_double, C.c_int, C.c_int, C.POINTER(StepInfo)]),
    "etp_step_batch": (C.c_int, [C.POINTER(_P), C.c_int, _D, _D, C.POINTER(StepInfo), C.POINTER(C.c_int)]),
    "etp_energy": (C.c_int, [_P, _D, _D, _D]),
    "etp_autotune": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "etp_krylov_method": (C.c_int, [_P, C.c_int]),
    "etp_newmark_step": (C.c_int, [_P, C.c_double, C.c_double, C.POINTER(C.c_int)]),
    "etp_state_get": (C.c_int, [_P, _D, _D, C.c_int]),
    "etp_state_set": (C.c_int, [_P, _D, _D, C.c_int]),
    "etp_state_upload": (C.c_int, [_P, _D, _D, C.c_int]),
    "etp_state_save": (C.c_int, [_P, C.c_char_p]),
    "etp_state_load": (C.c_int, [_P, C.c_char_p]),
    "etp_traj_steps": (C.c_int64, [_P]),
    "etp_apply_hbar": (C.c_int, [_P, C.c_int, _D, _D, _D]),
    "etp_apply_tangent": (C.c_int, [_P, _D, _D, _D]),
    "etp_expm_e1": (C.c_int, [_P, C.c_int, _D, C.c_double, _D]),
    "etp_expm_e1_noalloc": (C.c_int, [_P, C.c_int, _D, C.c_double, _D]),
    "etp_last_hessenberg": (C.c_int, [_P, C.POINTER(C.c_int), _D]),
    "etp_profile_enable": (C.c_int, [_P, C.c_int]),
    "etp_profile_read": (C.c_int, [_P, _I64, _D, _D, _D]),
    "etp_profile_reset": (C.c_int, [_P]),
    "etp_launch_count": (C.c_int64, [_P]),
    "etp_load_set": (C.c_int, [_P, _D]),
    "etp_traj_footprint": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "etp_batch_create": (C.c_int, [_P, C.c_size_t, C.c_int, C.POINTER(_P)]),
    "etp_batch_create_ragged": (C.c_int, [_P, C.c_size_t, C.POINTER(_P)]),
    "etp_batch_destroy": (None, [_P]),
    "etp_batch_admit": (C.c_int, [_P, _P, C.c_int, C.c_double, C.c_double]),
    "etp_batch_tick": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "etp_batch_retired": (C.c_int, [_P, C.POINTER(_P), C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]),
    "etp_batch_traj_info": (C.c_int, [_P, _P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), _F32,
                                      C.c_int, C.POINTER(C.c_int)]),
    "etp_batch_forget": (C.c_int, [_P, _P]),
    "etp_batch_usage": (C.c_int, [_P, C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
}

_lib = None


def lib():
    """Load libetp.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libetp.so not built ({LIB_PATH}); run paper_2405_05213_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != ETP_OK:
        raise EtpError(status, lib().etp_last_error().decode())
    return status


def _dptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _host_f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _dev_ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.cast(C.c_void_p(t.data_ptr()), _D)


# ------------------------------------------------------------------ C names
def etp_version():
    return lib().etp_version().decode()


def etp_ctx_create(device=0, stream=None):
    h = _P()
    _check(lib().etp_ctx_create(int(device), stream, C.byref(h)))
    return h


def etp_debug_spin_limit(ctx, polls):
    """Test hook: polls before a persistent-step barrier wait gives up (0 = built-in limit)."""
    _check(lib().etp_debug_spin_limit(ctx, int(polls)))


def etp_ctx_destroy(h):
    lib().etp_ctx_destroy(h)


def etp_mesh_create(ctx, order, coords, conn, fixed_dofs):
    coords = _host_f64(coords).reshape(-1, 3)
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    fixed = np.ascontiguousarray(fixed_dofs if fixed_dofs is not None else [], dtype=np.int32)
    h = _P()
    _check(lib().etp_mesh_create(ctx, int(order), coords.shape[0], _dptr(coords), conn.shape[0],
                                 conn.ctypes.data_as(_I32), fixed.size,
                                 fixed.ctypes.data_as(_I32) if fixed.size else None, C.byref(h)))
    return h


def etp_mesh_destroy(h):
    lib().etp_mesh_destroy(h)


def etp_material_set(mesh, kind, params, rho=1.0, elem_scale=None):
    p = _host_f64(params)
    es = None
    if elem_scale is not None:
        es_arr = np.ascontiguousarray(elem_scale, dtype=np.float32)
        es = es_arr.ctypes.data_as(_F32)
    _check(lib().etp_material_set(mesh, int(kind), _dptr(p), p.size, float(rho), es))


def etp_state_init(mesh, u0, v0, precision=ETP_PREC_FP64, m_cap=128):
    h = _P()
    if hasattr(u0, "is_cuda"):
        _check(lib().etp_state_init(mesh, _dev_ptr(u0), _dev_ptr(v0), 1, int(precision), int(m_cap), C.byref(h)))
    else:
        u = _host_f64(u0)
        v = _host_f64(v0, u.size)
        _check(lib().etp_state_init(mesh, _dptr(u), _dptr(v), 0, int(precision), int(m_cap), C.byref(h)))
    return h


def etp_traj_destroy(h):
    lib().etp_traj_destroy(h)


def etp_step(traj, dt, tol, m_fixed=0):
    m = C.c_int(0)
    e = C.c_double(0.0)
    _check(lib().etp_step(traj, float(dt), float(tol), int(m_fixed), C.byref(m), C.byref(e)))
    return m.value, e.value


def etp_step_ex(traj, dt, tol, m_fixed_pred=0, m_fixed_corr=0, check=True):
    info = StepInfo()
    st = lib().etp_step_ex(traj, float(dt), float(tol), int(m_fixed_pred), int(m_fixed_corr), C.byref(info))
    if check:
        _check(st)
    return st, info


def etp_step_batch(trajs, dts, tols, check=True):
    """One step of every trajectory in `trajs` (handles sharing one context)
    with its own dt and tol, as one ragged batch; returns (statuses, infos)."""
    n = len(trajs)
    hs = (_P * max(n, 1))(*[t for t in trajs])
    dt = (C.c_double * max(n, 1))(*[float(x) for x in dts])
    tl = (C.c_double * max(n, 1))(*[float(x) for x in tols])
    infos = (StepInfo * max(n, 1))()
    sts = (C.c_int * max(n, 1))()
    st = lib().etp_step_batch(hs, n, dt, tl, infos, sts)
    if check:
        _check(st)
    return [int(sts[i]) for i in range(n)], [infos[i] for i in range(n)]


def etp_krylov_method(traj, method):
    """ETP_KRYLOV_ARNOLDI (default) or ETP_KRYLOV_LANCZOS_ENERGY (linear materials, no load)."""
    _check(lib().etp_krylov_method(traj, int(method)))


def etp_newmark_step(traj, dt, tol=1e-12):
    """One Newmark-beta step (beta 1/4, gamma 1/2; linear materials); returns the CG iterations."""
    it = C.c_int(0)
    _check(lib().etp_newmark_step(traj, float(dt), float(tol), C.byref(it)))
    return it.value


def etp_autotune(traj, reps=3):
    """Time candidate launch shapes on this trajectory and keep the fastest (process-wide);
    returns the number of shapes stored."""
    n = C.c_int(0)
    _check(lib().etp_autotune(traj, int(reps), C.byref(n)))
    return n.value


def etp_energy(traj):
    t, k, p = C.c_double(), C.c_double(), C.c_double()
    _check(lib().etp_energy(traj, C.byref(t), C.byref(k), C.byref(p)))
    return t.value, k.value, p.value


def etp_state_get(traj, n_dofs):
    u = np.empty(n_dofs)
    v = np.empty(n_dofs)
    _check(lib().etp_state_get(traj, _dptr(u), _dptr(v), 0))
    return u, v


def etp_state_get_device(traj, u_out, v_out):
    _check(lib().etp_state_get(traj, _dev_ptr(u_out), _dev_ptr(v_out), 1))


def etp_state_set(traj, u, v):
    if hasattr(u, "is_cuda"):
        _check(lib().etp_state_set(traj, _dev_ptr(u), _dev_ptr(v), 1))
    else:
        u = _host_f64(u)
        v = _host_f64(v, u.size)
        _check(lib().etp_state_set(traj, _dptr(u), _dptr(v), 0))


def etp_state_upload(traj, u, v):
    """Send this trajectory's state back (host arrays or CUDA tensors), keeping its history."""
    if hasattr(u, "is_cuda"):
        _check(lib().etp_state_upload(traj, _dev_ptr(u), _dev_ptr(v), 1))
    else:
        u = _host_f64(u)
        v = _host_f64(v, u.size)
        _check(lib().etp_state_upload(traj, _dptr(u), _dptr(v), 0))


def etp_state_get_into(traj, u_out, v_out):
    """Host read-back into caller-owned (e.g. pinned) float64 arrays."""
    _check(lib().etp_state_get(traj, _dptr(u_out), _dptr(v_out), 0))


def etp_state_save(traj, path):
    _check(lib().etp_state_save(traj, str(path).encode()))


def etp_state_load(traj, path):
    _check(lib().etp_state_load(traj, str(path).encode()))


def etp_traj_steps(traj):
    return int(lib().etp_traj_steps(traj))


def etp_apply_hbar(mesh, precision, x, ustar=None):
    x = _host_f64(x)
    u = _host_f64(ustar, x.size) if ustar is not None else None
    y = np.empty_like(x)
    _check(lib().etp_apply_hbar(mesh, int(precision), _dptr(x), _dptr(u), _dptr(y)))
    return y


def etp_apply_tangent(mesh, x, u):
    """y = M^-1/2 K_T(u) M^-1/2 x (FP64 host arrays), the consistent tangent of a nonlinear material."""
    x = _host_f64(x)
    u = _host_f64(u, x.size)
    y = np.empty_like(x)
    _check(lib().etp_apply_tangent(mesh, _dptr(x), _dptr(u), _dptr(y)))
    return y


def etp_expm_e1(ctx, H, tau):
    H = np.asfortranarray(H, dtype=np.float64)
    n = H.shape[0]
    y = np.empty(n)
    _check(lib().etp_expm_e1(ctx, n, H.ctypes.data_as(_D), float(tau), _dptr(y)))
    return y


def etp_expm_e1_noalloc(ctx, n, H_dev, tau, y_dev):
    """exp(tau H) e_1 with caller-owned device buffers and no device allocation.

    H_dev: contiguous float64 CUDA tensor holding the n x n matrix column-major;
    y_dev: float64 CUDA tensor of length n (output). n <= 64.
    """
    _check(lib().etp_expm_e1_noalloc(ctx, int(n), _dev_ptr(H_dev), float(tau), _dev_ptr(y_dev)))


def etp_last_hessenberg(traj):
    m = C.c_int(0)
    _check(lib().etp_last_hessenberg(traj, C.byref(m), None))
    if m.value <= 0:
        return np.zeros((0, 0))
    H = np.zeros((m.value + 1) * m.value)
    _check(lib().etp_last_hessenberg(traj, C.byref(m), _dptr(H)))
    return H.reshape(m.value, m.value + 1).T


def etp_profile_enable(ctx, enable=True):
    _check(lib().etp_profile_enable(ctx, 1 if enable else 0))


def etp_profile_read(ctx):
    n = ETP_NUM_KERNEL_CLASSES
    la = (C.c_int64 * n)()
    ms = (C.c_double * n)()
    by = (C.c_double * n)()
    fl = (C.c_double * n)()
    _check(lib().etp_profile_read(ctx, la, ms, by, fl))
    return {KERNEL_CLASSES[k]: {"launches": int(la[k]), "ms": float(ms[k]), "bytes": float(by[k]),
                                "flops": float(fl[k])} for k in range(n)}


def etp_profile_reset(ctx):
    _check(lib().etp_profile_reset(ctx))


def etp_launch_count(ctx):
    return int(lib().etp_launch_count(ctx))


def etp_load_set(traj, P=None):
    """Constant external nodal forces (3*n_nodes, host), or None to remove the load."""
    if P is None:
        _check(lib().etp_load_set(traj, None))
    else:
        P = _host_f64(P)
        _check(lib().etp_load_set(traj, _dptr(P)))


def etp_traj_footprint(mesh, precision, m_cap):
    """(trajectory bytes, mesh bytes) of a trajectory etp_state_init would create."""
    tb, mb = C.c_size_t(0), C.c_size_t(0)
    _check(lib().etp_traj_footprint(mesh, int(precision), int(m_cap), C.byref(tb), C.byref(mb)))
    return int(tb.value), int(mb.value)


def etp_batch_create(ctx, device_budget_bytes, n_workers):
    h = _P()
    _check(lib().etp_batch_create(ctx, int(device_budget_bytes), int(n_workers), C.byref(h)))
    return h


def etp_batch_create_ragged(ctx, device_budget_bytes):
    h = _P()
    _check(lib().etp_batch_create_ragged(ctx, int(device_budget_bytes), C.byref(h)))
    return h


def etp_batch_destroy(h):
    lib().etp_batch_destroy(h)


def etp_batch_admit(batch, traj, n_steps, dt, tol):
    """True if admitted, False if the budget is full now (ETP_ERR_OOM)."""
    st = lib().etp_batch_admit(batch, traj, int(n_steps), float(dt), float(tol))
    if st == ETP_ERR_OOM:
        return False
    _check(st)
    return True


def etp_batch_tick(batch):
    n = C.c_int(0)
    _check(lib().etp_batch_tick(batch, C.byref(n)))
    return n.value


def etp_batch_retired(batch, max_n=256):
    trajs = (_P * max_n)()
    sts = (C.c_int * max_n)()
    n = C.c_int(0)
    _check(lib().etp_batch_retired(batch, trajs, sts, int(max_n), C.byref(n)))
    return [(trajs[i], int(sts[i])) for i in range(n.value)]


def etp_batch_traj_info(batch, traj):
    """(steps done, status, retired, per-step host ms as a numpy array)."""
    sd, st, rt, n = C.c_int(0), C.c_int(0), C.c_int(0), C.c_int(0)
    _check(lib().etp_batch_traj_info(batch, traj, C.byref(sd), C.byref(st), C.byref(rt), None, 0, C.byref(n)))
    ms = np.zeros(max(n.value, 1), dtype=np.float32)
    _check(lib().etp_batch_traj_info(batch, traj, C.byref(sd), C.byref(st), C.byref(rt),
                                     ms.ctypes.data_as(_F32), int(n.value), C.byref(n)))
    return sd.value, st.value, bool(rt.value), ms[:n.value].copy()


def etp_batch_forget(batch, traj):
    _check(lib().etp_batch_forget(batch, traj))


def etp_batch_usage(batch):
    r, n = C.c_size_t(0), C.c_int(0)
    _check(lib().etp_batch_usage(batch, C.byref(r), C.byref(n)))
    return int(r.value), n.value


# ------------------------------------------------------------------ owners
class Context:
    def __init__(self, device=0, stream=None):
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except ImportError:
                stream = None
        self.stream = stream
        self.h = etp_ctx_create(device, C.c_void_p(stream) if stream else None)

    def close(self):
        if self.h:
            etp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx, order, coords, conn, fixed_dofs):
        self.ctx = ctx
        self.n_nodes = int(np.asarray(coords).reshape(-1, 3).shape[0])
        self.h = etp_mesh_create(ctx.h, order, coords, conn, fixed_dofs)

    @classmethod
    def from_problem(cls, ctx, prob):
        m = cls(ctx, prob.mesh.order, prob.mesh.coords, prob.mesh.conn, prob.fixed_dofs)
        m.set_material(prob.material, prob.params, prob.rho, prob.elem_scale)
        return m

    @property
    def n_dofs(self):
        return 3 * self.n_nodes

    def set_material(self, kind, params, rho=1.0, elem_scale=None):
        etp_material_set(self.h, kind, params, rho, elem_scale)

    def apply_hbar(self, x, ustar=None, precision=ETP_PREC_FP64):
        return etp_apply_hbar(self.h, precision, x, ustar)

    def close(self):
        if self.h:
            etp_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Trajectory:
    def __init__(self, mesh, u0, v0, precision=ETP_PREC_FP64, m_cap=128):
        self.mesh = mesh
        self.h = etp_state_init(mesh.h, u0, v0, precision, m_cap)

    def step(self, dt, tol, m_fixed=0):
        return etp_step(self.h, dt, tol, m_fixed)

    def step_ex(self, dt, tol, m_fixed_pred=0, m_fixed_corr=0, check=True):
        return etp_step_ex(self.h, dt, tol, m_fixed_pred, m_fixed_corr, check)

    def energy(self):
        return etp_energy(self.h)

    def set_krylov(self, method):
        etp_krylov_method(self.h, method)

    def state(self):
        return etp_state_get(self.h, self.mesh.n_dofs)

    def set_state(self, u, v):
        etp_state_set(self.h, u, v)

    def set_load(self, P=None):
        etp_load_set(self.h, P)

    def save(self, path):
        etp_state_save(self.h, path)

    def load(self, path):
        etp_state_load(self.h, path)

    @property
    def steps(self):
        return etp_traj_steps(self.h)

    def last_hessenberg(self):
        return etp_last_hessenberg(self.h)

    def close(self):
        if self.h:
            etp_traj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
