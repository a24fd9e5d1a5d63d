// Host-side helpers shared by the translation units of libetp.
#pragma once

#include <string>
#include <vector>

#include "etp_internal.cuh"
#include "fe_kernels.cuh"

namespace etp {

// Device allocation with the library's error reporting; dfree tolerates null.
template <typename P>
inline etp_status dalloc(P** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) return ETP_OK;
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ETP_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return ETP_OK;
}

template <typename P>
inline void dfree(P*& ptr) {
  if (ptr) cudaFree((void*)ptr);
  ptr = nullptr;
}

// Event-bracketed launch accounting (CUDA events on the context stream).
struct ProfScope {
  etp_ctx* ctx;
  int cls;
  double bytes;
  double flops;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(etp_ctx* c, int k, double by, double fl = 0.0);
  ~ProfScope();
};

cudaEvent_t take_event(etp_ctx* ctx);

template <int P, typename T>
cudaError_t launch_elem_apply(const ApplyParams<T>& p, int kind, bool box, int ns, int num_sms, cudaStream_t st,
                              int grid);
template <int P, typename T>
cudaError_t launch_frozen_build(const FrozenBuildParams<T>& p, int kind, bool box, cudaStream_t st);

// Stored frozen coefficients of fz's states (count of them) into bufs[k]
// (frozen_nf(kind) x n_elems x nq elements of T each); sets fz.data. An
// inverted Gauss point sets KERR_INVERTED in *err.
template <typename T>
etp_status build_frozen(etp_mesh* m, FrozenSet& fz, void* const* bufs, int* err);

// Bytes of one stored frozen-coefficient buffer of mesh m in precision size s.
size_t frozen_buffer_bytes(const etp_mesh* m, size_t s);

// Device bytes of a mesh and of one trajectory on it (what etp_state_init allocates).
size_t mesh_device_bytes(const etp_mesh* m);
size_t traj_device_bytes(const etp_mesh* m, int precision, int m_cap);

// Operator apply z = A x for a Krylov vector x of the trajectory's precision:
// element pass and node gather. Nonlinear materials need fz.data (build_frozen).
// `stop` may be null.
// `pbar` (SoA 3*nn_pad, or null): constant external load P_bar, multiplied by
// the augmented entry of x (row 3*nn_pad - 1) in the velocity rows.
// kind_override >= 0 applies another operator kind with the same stored
// fields (MAT_SVK_TANGENT on SVK coefficients).
template <typename T>
etp_status apply_A(etp_mesh* m, const T* x, const double* xscale, const FrozenSet& fz, T* Ye, T* z,
                   const int* stop, const T* pbar = nullptr, bool gather = true, int kind_override = -1);

// One Krylov solve: w_out = exp(tau A) w_in (Section 4.3).
struct SolveResult {
  int m = 0;
  double eps = 0.0;
  double beta = 0.0;
  bool converged = false;
};
etp_status krylov_solve(etp_traj* t, double tau, const double* w_in, double* w_out, const FrozenSet& fz,
                        double tol, int m_fixed, void* ustar_out, SolveResult* res, int kind);

etp_status run_expm_window(etp_ctx* ctx, const double* H, int ldH, int j0, int j1, double tau, double* ws, int ld,
                           int* s_arr, const KState* ks, int* h_s);

// Bytes of per-tile partial sums of the persistent Arnoldi step (solve.cu).
size_t pk_partials_bytes(int64_t L, int m_cap, int precision);

// Stored frozen coefficients of fz's states for a solve of trajectory t
// (reused per midpoint-history slot while unchanged); fzb gets the data pointers.
template <typename T>
etp_status prepare_frozen(etp_traj* t, const FrozenSet& fz, FrozenSet* fzb);

// Element-pass parameters of z = A x for mesh m (apply_A's launch arguments),
// and the pass's algorithmic bytes and flops with ns frozen states.
template <typename T>
ApplyParams<T> make_apply_params(const etp_mesh* m, const T* x, const double* xscale, const FrozenSet& fz, T* Ye,
                                 const int* stop);
double elem_apply_bytes(const etp_mesh* m, int ns, size_t s);
double elem_apply_flops_of(const etp_mesh* m, int ns);
template <int P, typename T>
cudaError_t launch_elem_apply_batch(ElemBatch<T>& b, int kind, bool box, int ns, int num_sms, cudaStream_t st);

// Pieces of one time step shared by etp_step_ex and etp_step_batch (api.cu).
etp_status check_step_args(const etp_traj* t, double dt, double tol);
etp_status predictor_setup(etp_traj* t, FrozenSet* fp, int* slot_new);
FrozenSet corrector_frozen(const etp_traj* t, int slot_new);
etp_status step_commit(etp_traj* t, const SolveResult& rc, int slot_new, etp_step_info* loc, etp_step_info* info);

// Iteration-level continuous batching of Krylov solves (batch_solve.cu): the
// engine behind etp_step_batch and the ragged serving batch. Trajectories are
// added with a number of steps; each tick advances every active solve by one
// Arnoldi step in batched launches and reports each finished step.
struct RaggedEngine;
struct EngineEvent {
  etp_traj* t;
  etp_status st;       // status of the finished step (not committed unless ETP_OK)
  etp_step_info info;
  bool last;           // the trajectory left the engine (all steps done, or failed)
};
RaggedEngine* ragged_engine_create(etp_ctx* ctx);
void ragged_engine_destroy(RaggedEngine* e);
bool ragged_engine_empty(const RaggedEngine* e);
etp_status ragged_engine_add(RaggedEngine* e, etp_traj* t, double dt, double tol, int n_steps);
etp_status ragged_engine_tick(RaggedEngine* e, std::vector<EngineEvent>* events);

// Whole-solve cooperative kernel for short vectors on Q1 boxes
// (solve_fused_f{32,64}.cu): the plan of one launch (the last Arnoldi step it
// can reach within cap, 0: not available; grid; dynamic shared memory and its
// partial-sum copy area) and the launch.
template <typename T>
struct FusedSolve;
struct FusedPlan {
  int j_end = 0;
  int grid = 0;
  size_t dyn = 0;
  uint32_t red_off = 0, red_bytes = 0;
};
template <typename T>
FusedPlan fused_plan(int kind, int ns, int cap, int64_t L, int num_sms);
template <typename T>
cudaError_t launch_fused_solve(etp_ctx* ctx, const FusedSolve<T>& f, int kind, int ns, const FusedPlan& plan);

// Bytes of the Newmark-beta workspace of a trajectory (newmark.cu).
size_t newmark_work_bytes(const etp_traj* t);

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace etp
