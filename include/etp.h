/*
 * etp.h - C ABI of libetp, a GB300 (sm_103a) implementation of the exponential
 * time propagator for elastodynamics of arXiv 2405.05213.
 *
 * One call of etp_step advances the state w_bar = [M^{1/2} u; M^{1/2} v] of the
 * first-order recast (Section 2.3, Eq. "A expression at P=0") by one time step
 * of the first Magnus term (Section 3, Eqs. "truncOmegaB", "quadratureApprox"):
 *     w_bar_n = exp(dt A(u_mid)) w_bar_{n-1},   A = [[0, I], [-H_bar(u), 0]],
 * with exp(dt A) w evaluated by Arnoldi (Section 4.3) and the subspace size m
 * chosen by the a-priori estimate (Eq. "subspace error estimate"). Nonlinear
 * materials use the predictor-corrector of Section 4.2.
 *
 * Conventions shared by every call:
 *  - Status: every call returns etp_status; ETP_OK is 0. After a non-OK status
 *    etp_last_error() returns a message for the calling thread.
 *  - Ownership: each *_create returns a handle owned by the caller and released
 *    by the matching *_destroy. Host arrays passed in are copied; the caller keeps
 *    them. Device memory is allocated by the library (cudaMalloc) and released by
 *    the *_destroy calls. A mesh must outlive its trajectories; a context must
 *    outlive its meshes.
 *  - Streams: all device work of a context runs on the CUDA stream given to
 *    etp_ctx_create (0 = the legacy default stream). Calls that return host
 *    results synchronise that stream.
 *  - Layout of user vectors: node-major, 3 components per node, global DOF
 *    index 3*node + comp, FP64, length 3*n_nodes. Nodes are numbered 0..n_nodes-1.
 *  - Element connectivity: lexicographic local order, local node
 *    a + (p+1)*(b + (p+1)*c) sits at reference coordinates
 *    (-1 + 2a/p, -1 + 2b/p, -1 + 2c/p) for polynomial order p.
 *  - Dirichlet DOFs (u = 0, Section 2.1) are eliminated: the state stays zero there.
 */
#ifndef ETP_H
#define ETP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct etp_ctx etp_ctx;
typedef struct etp_mesh etp_mesh;
typedef struct etp_traj etp_traj;

typedef enum {
  ETP_OK = 0,
  ETP_ERR_INVALID = 1,          /* bad argument or call order */
  ETP_ERR_OOM = 2,              /* device allocation failed */
  ETP_ERR_CUDA = 3,             /* CUDA runtime error */
  ETP_ERR_NOT_CONVERGED = 4,    /* estimate above tol at m_cap; state not advanced */
  ETP_ERR_NONFINITE = 5,        /* NaN/Inf in the state or in the Krylov process */
  ETP_ERR_INVERTED_ELEMENT = 6, /* det F <= 0 at a Gauss point of the frozen state */
  ETP_ERR_TIMEOUT = 7,          /* a bounded device-side wait gave up; step not committed */
  ETP_ERR_IO = 8                /* checkpoint file error */
} etp_status;

/* FP64: every vector and reduction in FP64.
 * MIXED: operator apply and Krylov basis in FP32; Gram-Schmidt coefficients,
 * norms, the Hessenberg matrix, its exponential and the state w_bar in FP64. */
typedef enum { ETP_PREC_FP64 = 0, ETP_PREC_MIXED = 1 } etp_precision;

/* Materials and their params (in this order):
 *   LINEAR         {E, nu}              small-strain isotropic elasticity, H = K
 *   NEOHOOKE       {mu, lambda}         psi = mu/2 (I1-3) - mu ln J + lambda/2 (ln J)^2
 *   MOONEY_RIVLIN  {C10, C01, kappa}    psi = C10 (I1b-3) + C01 (I2b-3) + kappa/2 (J-1)^2
 *   SVK            {lambda, mu}         Appendix A.1
 *   YEOH           {C10, C20, C30, D1}  Appendix A.2
 * The nonlinear H(u*) is the frozen-coefficient secant split with
 * H(u*) u* = R(u*) (Section 2.3, Appendix A): P_lin(G) = F* S_lin(G), with
 * E_lin(G) = sym(G) + sym(D*^T G)/2 and j_lin(G) = P_e(D*) : G (Appendix A.2). */
typedef enum {
  ETP_MAT_LINEAR = 0,
  ETP_MAT_NEOHOOKE = 1,
  ETP_MAT_MOONEY_RIVLIN = 2,
  ETP_MAT_SVK = 3,
  ETP_MAT_YEOH = 4
} etp_material_kind;

/* Per-solve report of one etp_step_ex call. */
typedef struct {
  int m_pred;          /* Krylov size of the predictor solve (0 for linear) */
  int m_corr;          /* Krylov size of the corrector (the only solve for linear) */
  double eps_pred;     /* a-priori estimate eps_m of each solve (absolute) */
  double eps_corr;
  double beta;         /* ||w_bar_{n-1}|| */
  int converged;       /* 1 if every solve met eps_m <= tol * ||w|| (or broke down) */
} etp_step_info;

/* Message for the last non-OK status returned to this thread ("" if none). */
const char* etp_last_error(void);

/* Library version string. */
const char* etp_version(void);

/* Every device-side wait of the library is bounded (the paper has no
 * counterpart; this is how the runtime reports a stuck step instead of hanging
 * the GPU). A grid-barrier wait of the persistent Arnoldi step, a barrier of the
 * cooperative a-priori check or a bulk-copy wait that gives up records the
 * failure on the device; the kernel still ends, the call returns
 * ETP_ERR_TIMEOUT, the step is not committed (state, history and step count
 * unchanged) and the barrier words are reset, so the next step of the same
 * trajectory runs normally.
 *
 * Test hook: etp_debug_spin_limit sets how many polls a grid-barrier wait of
 * the persistent Arnoldi step (vectors of up to 2^20 rows) makes before it
 * gives up, for the steps of this context that follow; 0 restores the built-in
 * limit (2^23 polls, seconds). A low limit makes the wait run out, so a test can
 * check the ETP_ERR_TIMEOUT path: the step computes wrong values in that case
 * but every index stays in bounds and every block ends. While a lower limit is
 * set, solves step with one launch per Arnoldi step (the whole-solve kernel,
 * whose check stages read loop counts from the device, is not used). Other
 * waits keep their built-in limits. Returns ETP_ERR_INVALID for a null context. */
etp_status etp_debug_spin_limit(etp_ctx* ctx, uint64_t polls);

/* Context on CUDA device `device`; `cuda_stream` is a cudaStream_t (may be NULL). */
etp_status etp_ctx_create(int device, void* cuda_stream, etp_ctx** out);
void etp_ctx_destroy(etp_ctx* ctx);

/* Mesh of hexahedra (Section 2.2, Eq. "expansion in finite-element basis").
 *   order       1 (8-node Q1) or 2 (27-node Q2)
 *   coords      host, n_nodes*3 FP64, reference-configuration positions
 *   conn        host, n_elems*(order+1)^3 int32, lexicographic local order
 *   fixed_dofs  host, n_fixed int32 global DOF ids 3*node+comp (may be NULL if 0)
 * Elements with det J <= 0 at a quadrature point are rejected (ETP_ERR_INVALID).
 * Structured uniform boxes (the layout of a lexicographic box generator) are
 * detected and use constant element geometry. */
etp_status etp_mesh_create(etp_ctx* ctx, int order, int64_t n_nodes, const double* coords,
                           int64_t n_elems, const int32_t* conn, int64_t n_fixed,
                           const int32_t* fixed_dofs, etp_mesh** out);
void etp_mesh_destroy(etp_mesh* mesh);

/* Material law, density and optional per-element stiffness scale (host,
 * n_elems floats, multiplies the stress; NULL = 1). Computes the diagonal GLL
 * mass (Section 2.2) on the device. Must precede etp_state_init. */
etp_status etp_material_set(etp_mesh* mesh, int kind, const double* params, int n_params,
                            double rho, const float* elem_scale);

/* Trajectory: state u0, v0 (length 3*n_nodes FP64; host pointers if
 * on_device == 0, device pointers otherwise), precision (etp_precision) and
 * the Krylov capacity m_cap (1..256). Allocates (m_cap+1) basis vectors. */
etp_status etp_state_init(etp_mesh* mesh, const double* u0, const double* v0, int on_device,
                          int precision, int m_cap, etp_traj** out);
void etp_traj_destroy(etp_traj* traj);

/* One time step of size dt. tol is relative: a solve stops at the smallest m
 * with eps_m <= tol * ||w_bar|| (Eq. "subspace error estimate"). m_fixed > 0
 * skips the test and uses m = m_fixed (Section 6.2 fixes m for a run); a happy
 * breakdown (h_{m+1,m} <= 1e-14 ||H_m||_F) ends a solve early with the exact
 * result. m_out / err_out (nullable) receive the corrector's m and eps.
 * On ETP_ERR_NOT_CONVERGED the state is left at w_bar_{n-1}. */
etp_status etp_step(etp_traj* traj, double dt, double tol, int m_fixed, int* m_out, double* err_out);

/* As etp_step with separate fixed sizes for the predictor and corrector solves
 * (0 = adaptive for that solve) and a full report (nullable). */
etp_status etp_step_ex(etp_traj* traj, double dt, double tol, int m_fixed_pred, int m_fixed_corr,
                       etp_step_info* info);

/* Ragged batched step: one etp_step_ex(dt[i], tol[i], adaptive m) of each of
 * the n (0..64) trajectories trajs[i], which may differ in mesh, size, order,
 * material, precision, dt and tol but must share one context (its stream runs
 * the batch) and appear once each. Their Krylov solves (Section 4.3; the
 * predictor and corrector of Section 4.2) advance with iteration-level
 * batching: each Arnoldi step of all active solves is one element-pass launch
 * per (order, precision, material, geometry, frozen-state count) class and one
 * cooperative persistent-step launch per precision and tile size for up to 16
 * trajectories; the a-priori checks due at a step share one batched
 * small-exponential launch set and two host synchronisations; a trajectory
 * starts its corrector as soon as its predictor selects m. Vectors of more than
 * 2^20 rows are stepped by etp_step_ex. A trajectory's result is bitwise the
 * same as from etp_step_ex alone.
 * infos / statuses (nullable, n entries) receive each trajectory's report and
 * status; a trajectory whose step failed is left at w_bar_{n-1}, the others
 * are committed. Returns ETP_OK, the first failing trajectory's status, or
 * ETP_ERR_INVALID (bad arguments: nothing is stepped) / ETP_ERR_CUDA. */
etp_status etp_step_batch(etp_traj* const* trajs, int n, const double* dt, const double* tol,
                          etp_step_info* infos, etp_status* statuses);

/* Newmark-beta step (beta = 1/4, gamma = 1/2), the comparison integrator of
 * Section 6, for every material with P = 0, in the mass-scaled variables.
 * LINEAR: (I + beta dt^2 H_bar) a_new = -H_bar u_pred by conjugate gradients
 * warm-started from the previous acceleration. Nonlinear materials ("fully
 * implicit"): Newton iterations on a + R_bar(u_pred + beta dt^2 a) = 0 from the
 * previous acceleration, the residual through the secant identity
 * H(u) u = R(u), each correction by CG with the consistent tangent dP/dF (SVK
 * in closed form; Neo-Hooke, Mooney-Rivlin and Yeoh as the exact directional
 * derivative of P(F) = F S(C) in dual-number arithmetic); stop
 * when ||residual|| <= tol ||a|| (at most 30 iterations). CG: relative residual
 * <= tol, checked every 4 iterations (iterations past convergence only
 * refine; one host synchronisation per check, none at the end of the step:
 * the call returns with the step's last kernels queued on the context stream),
 * at most 20000. tol in (0,1). FP64 matrix-free operators throughout.
 * Works on the trajectory's own state (etp_energy / etp_state_get read it; the
 * acceleration is recomputed from the state after any other change of it).
 * The first call allocates an FP64 workspace of about 4.5 state vectors plus
 * the element terms (and the stored coefficients of the Newton iterate).
 * *iters_out (nullable) = CG iterations of the step. ETP_ERR_INVALID for a load;
 * ETP_ERR_NOT_CONVERGED (state unchanged) if CG or Newton does not converge. */
etp_status etp_newmark_step(etp_traj* traj, double dt, double tol, int* iters_out);

/* Autotuner (launch shapes only; the paper has no counterpart): times, on
 * this trajectory's own buffers, `reps` launches of every candidate tile shape
 * of the Gram-Schmidt passes (rows per tile, pipeline stages, blocks per SM;
 * probed column counts up to m_cap, vectors longer than 2^20 rows) and every
 * candidate grid of the Q1 element pass, and keeps the fastest for every
 * trajectory of the same precision and vector length (element pass: same
 * order, material, geometry and element count), process-wide.
 * *n_configs (nullable) = shapes stored. Overwrites the Krylov workspace, not
 * the state: call between steps. Element results do not depend on the grid;
 * Gram-Schmidt results change at rounding level with the tile shape (partial
 * sums are grouped per block). reps in 1..100. */
etp_status etp_autotune(etp_traj* traj, int reps, int* n_configs);

/* Krylov process of a trajectory's solves (Section 4.3).
 *   ETP_KRYLOV_ARNOLDI (default): Arnoldi with CGS2 in the Euclidean inner
 *     product, as the paper; every material, with or without load.
 *   ETP_KRYLOV_LANCZOS_ENERGY: for LINEAR materials without load, H_bar is
 *     symmetric positive definite and A = [[0, I], [-H_bar, 0]] is skew-adjoint in
 *     the energy inner product <w, w'>_E = u^T H_bar u' + v^T v' (Section 5.2,
 *     Eq. "energyExpr"), so Arnoldi in that inner product reduces to a
 *     three-term (Lanczos) recurrence with a skew-symmetric tridiagonal T_m:
 *     one apply, one axpy pass and one two-term dot pass per Krylov step instead
 *     of two Gram-Schmidt passes over all previous columns. The estimate and
 *     the tolerance are those of etp_step measured in the energy norm:
 *     eps_m = tau beta_m ||w||_E |[exp(tau T_m)]_{m,1}| <= tol ||w||_E. The
 *     basis is not reorthogonalised (the approximation of exp(tau A) w by the
 *     Lanczos process stays accurate as orthogonality fades).
 * Errors: ETP_ERR_INVALID for an unknown method, or Lanczos on a nonlinear
 * material; a step with a load set returns ETP_ERR_INVALID (not committed). */
enum { ETP_KRYLOV_ARNOLDI = 0, ETP_KRYLOV_LANCZOS_ENERGY = 1 };
etp_status etp_krylov_method(etp_traj* traj, int method);

/* Energy (Section 5.2, Eq. "energyExpr"): kinetic v_bar^T v_bar / 2 and
 * potential sum_e sum_q psi(F) w detJ (equal to u_bar^T H_bar u_bar / 2 for
 * LINEAR), minus P^T u when a constant load is set (etp_load_set). Any
 * pointer may be NULL. */
etp_status etp_energy(etp_traj* traj, double* total, double* kinetic, double* potential);

/* Physical displacement and velocity (3*n_nodes FP64). on_device selects
 * device or host pointers. Either pointer may be NULL. */
etp_status etp_state_get(etp_traj* traj, double* u_out, double* v_out, int on_device);
/* Replace the state (same layout); resets the predictor history. */
etp_status etp_state_set(etp_traj* traj, const double* u, const double* v, int on_device);
/* Upload the state of this same trajectory (same layout) and keep its
 * predictor history and step count: for a caller that keeps the state in host
 * memory between steps and sends it back before each step. */
etp_status etp_state_upload(etp_traj* traj, const double* u, const double* v, int on_device);

/* Constant external load P (Section 2.3, Eq. "A expression at P != 0"): the
 * state becomes [u_bar; v_bar; 1] and A gains the column P_bar = M^{-1/2} P in
 * the velocity rows, so exp(dt A) propagates forced motion exactly for a load
 * constant over the step. P: host, 3*n_nodes physical nodal forces
 * (node-major, 3*node+comp; components on fixed DOFs are ignored); copied.
 * NULL removes the load. The augmented entry lives in a padding row of the
 * device state (every mesh has at least one padding node), the Krylov
 * tolerance is relative to the norm of the augmented state as in the paper,
 * and etp_energy adds the load potential -P^T u to the potential energy (the
 * conserved total of a conservative load). The load is not part of a
 * checkpoint: set it again after etp_state_load. Errors: ETP_ERR_INVALID for
 * a non-finite entry, ETP_ERR_OOM. */
etp_status etp_load_set(etp_traj* traj, const double* P);

/* Checkpoint: w_bar (FP64), step index and the predictor history, so that a
 * resumed run continues bit-identically. */
etp_status etp_state_save(etp_traj* traj, const char* path);
etp_status etp_state_load(etp_traj* traj, const char* path);

/* Number of steps taken. */
int64_t etp_traj_steps(const etp_traj* traj);

/* ---------------------------------------------------------------- kernels
 * Single-kernel entry points of the step, for checking and benchmarking.
 * Host pointers unless stated otherwise. */

/* y = H_bar(u*) x on the full DOF vector (Section 2.3: M^{-1/2} H(u*) M^{-1/2}),
 * with Dirichlet entries of y set to 0. x, ustar, y: 3*n_nodes FP64 host.
 * ustar may be NULL (u* = 0; required for LINEAR). precision as etp_precision. */
etp_status etp_apply_hbar(etp_mesh* mesh, int precision, const double* x, const double* ustar,
                          double* y);

/* y = M^{-1/2} K_T(u) M^{-1/2} x with K_T = dR/du the consistent tangent of the
 * internal force at displacement u (Section 2.1, S = dpsi/dE; the operator of
 * the Newton corrections of the fully implicit Newmark-beta step, Section 6),
 * FP64, Dirichlet entries of y set to 0. x, u, y: 3*n_nodes FP64 host.
 * Nonlinear materials only (ETP_ERR_INVALID for LINEAR, where K_T = K and
 * etp_apply_hbar applies it). */
etp_status etp_apply_tangent(etp_mesh* mesh, const double* x, const double* u, double* y);

/* y = exp(tau * H) e_1 for an n x n FP64 matrix H (host, column-major), with the
 * GPU small-exponential kernels of the Krylov step (Section 4.3: Taylor series
 * after scaling by 2^-s, then s squarings). n <= 256. */
etp_status etp_expm_e1(etp_ctx* ctx, int n, const double* H, double tau, double* y);

/* Allocation-free variant of etp_expm_e1 (the paper has no counterpart; this
 * is a library service). For callers that cannot allocate device memory:
 * real-time loops in which cudaMalloc could stall or synchronise the device,
 * processes that fix their device-memory budget at start-up, or hosts whose
 * device memory is handed out by another allocator as fixed buffers.
 *   H  device pointer, n x n FP64, column-major (input, caller-owned)
 *   y  device pointer, n FP64 (output, caller-owned): exp(tau * H) e_1
 *   n  1..64; larger n returns ETP_ERR_INVALID.
 * The workspace is one static device array of 6*64*64+32 doubles (~192 KiB)
 * that every GPU which loads the library holds until the process exits; the
 * call allocates and frees nothing. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current: make
 * that first call before any stream capture. All calls on a device share the
 * one array, so calls that overlap on the GPU (other streams, other threads)
 * race; each call writes every workspace entry before reading it, so nothing
 * carries over from the previous call. Runs on the context's stream and
 * synchronises it twice (to read the scaling exponent, and at the end). */
etp_status etp_expm_e1_noalloc(etp_ctx* ctx, int n, const double* H, double tau, double* y);

/* Copies of the last Krylov solve's Hessenberg matrix ((m+1) x m, column-major
 * FP64 host, leading dimension m+1) and its size m. H may be NULL to query m. */
etp_status etp_last_hessenberg(etp_traj* traj, int* m, double* H);

/* ---------------------------------------------------------------- serving
 * Continuous batching of trajectories (the served mixed batch). The paper
 * propagates one trajectory at a time and has no counterpart; this is the
 * runtime around the propagator for many concurrent requests.
 *
 * Device footprint of a trajectory etp_state_init would create on `mesh` with
 * this precision and m_cap, and of the mesh itself (bytes; either pointer may
 * be NULL). Used for admission before anything is allocated. */
etp_status etp_traj_footprint(const etp_mesh* mesh, int precision, int m_cap, size_t* traj_bytes,
                              size_t* mesh_bytes);

typedef struct etp_batch etp_batch;
/* A batch with a device-memory budget (bytes) and n_workers host threads
 * (1..256) that step the admitted trajectories. Trajectories on different
 * contexts step concurrently (their kernels overlap on the GPU); two of one
 * context never do. The batch does not own the trajectories. */
etp_status etp_batch_create(etp_ctx* ctx, size_t device_budget_bytes, int n_workers, etp_batch** out);
/* Ragged batch: the admitted trajectories of each context are run by one
 * worker with iteration-level continuous batching (the engine of
 * etp_step_batch) on that context's stream: each tick advances every active
 * Krylov solve of the context by one Arnoldi step in shared launches, a
 * trajectory moves to its next solve as soon as one selects m, and requests
 * admitted meanwhile join at the next tick. Trajectories of different
 * contexts run in separate engines whose kernels overlap on the GPU (a worker
 * starts with the first admitted trajectory of a context and ends when none of
 * the context's trajectories is left in the batch). The
 * other etp_batch_* calls behave as for etp_batch_create; the recorded time of
 * a step is the wall time since the trajectory's previous step finished (or
 * it joined). Each trajectory's result is bitwise the same as stepped alone. */
etp_status etp_batch_create_ragged(etp_ctx* ctx, size_t device_budget_bytes, etp_batch** out);
/* Joins the workers (a step in flight completes first). Trajectories stay
 * valid and owned by the caller. */
void etp_batch_destroy(etp_batch* batch);
/* Admit `traj` for n_steps steps of etp_step(dt, tol, adaptive m). Its
 * footprint (trajectory + mesh) is reserved against the budget; ETP_ERR_OOM
 * means "not now" (retry after a tick has retired something); ETP_ERR_INVALID
 * for bad arguments or a trajectory already admitted. Stepping starts at once
 * on a free worker. */
etp_status etp_batch_admit(etp_batch* batch, etp_traj* traj, int n_steps, double dt, double tol);
/* Block until at least one step has finished since the previous tick (or no
 * admitted trajectory has work left); *n_finished_steps = steps completed
 * since then. Trajectories that completed their n_steps, or whose step failed
 * (the failed step is not committed: state at the last good step), are
 * retired: removed from the batch and from the budget, and queued for
 * etp_batch_retired. */
etp_status etp_batch_tick(etp_batch* batch, int* n_finished_steps);
/* Collect up to max retired trajectories (in retirement order) and their final
 * status (ETP_OK or the failing step's status); *n = how many. */
etp_status etp_batch_retired(etp_batch* batch, etp_traj** trajs, int* statuses, int max, int* n);
/* Steps done, status, retired flag and the host wall time (ms) of every step
 * of an admitted or retired trajectory: up to max_ms values into step_ms
 * (*n_ms = count written; with step_ms NULL, *n_ms = steps recorded). */
etp_status etp_batch_traj_info(etp_batch* batch, const etp_traj* traj, int* steps_done, int* status,
                               int* retired, float* step_ms, int max_ms, int* n_ms);
/* Drop the record of a retired trajectory (before destroying it). */
etp_status etp_batch_forget(etp_batch* batch, const etp_traj* traj);
/* Bytes reserved by admitted trajectories and their number. */
etp_status etp_batch_usage(etp_batch* batch, size_t* reserved_bytes, int* n_active);

/* ---------------------------------------------------------------- profiling
 * Per-kernel-class CUDA-event timing of launches made by etp_step while enabled.
 * Classes: 0 element apply, 1 node gather, 2 CGS dot, 3 CGS update+dot,
 * 4 CGS update+norm, 5 small exponential, 6 state combine, 7 other,
 * 8 fused Arnoldi step (node gather and the three CGS2 passes in one
 * persistent launch, used for vectors of up to 2^20 rows), 9 frozen-state
 * coefficients (once per Krylov solve and frozen state: grad u* and the
 * material factors at every Gauss point), 10 Lanczos vector passes (the
 * three-term update and the energy-norm pass of ETP_KRYLOV_LANCZOS_ENERGY). */
#define ETP_NUM_KERNEL_CLASSES 11
etp_status etp_profile_enable(etp_ctx* ctx, int enable);
/* Synchronises; per class: launches, total milliseconds, algorithmic bytes and
 * algorithmic flops (element apply and frozen-state coefficients: operation
 * count of the secant-stress formulation per Gauss point; other classes 0). Any array may be NULL. */
etp_status etp_profile_read(etp_ctx* ctx, int64_t* launches, double* ms, double* bytes, double* flops);
etp_status etp_profile_reset(etp_ctx* ctx);
/* Number of kernel launches made by this context since creation. */
int64_t etp_launch_count(const etp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* ETP_H */
