// Internal data structures and launch helpers of libetp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/etp.h"

namespace etp {

// --------------------------------------------------------------- errors
void set_error(const std::string& msg);
etp_status fail(etp_status s, const std::string& msg);

#define ETP_CUDA_TRY(call)                                                              \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess)                                                              \
      return ::etp::fail(ETP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

#define ETP_TRY(expr)                 \
  do {                                \
    etp_status _s = (expr);           \
    if (_s != ETP_OK) return _s;      \
  } while (0)

// Device error codes written by kernels into KState::err.
enum : int { KERR_NONE = 0, KERR_NONFINITE = 1, KERR_INVERTED = 2, KERR_TIMEOUT = 4 };

constexpr int kMaxQ = 27;     // quadrature points per element (Q2: 3x3x3)
constexpr int kMaxNen = 27;   // nodes per element
constexpr int kMaxParams = 8;
constexpr int kMaxCap = 256;  // largest Krylov capacity
constexpr int kCgsMaxBlocksPerSm = 8;  // grid cap of the Gram-Schmidt passes (x SM count)
constexpr int64_t kPkMaxRows = (int64_t)1 << 20;  // vectors up to this length use the persistent step
constexpr int kMaxCand = 64;  // candidate Krylov sizes checked by one small-exponential launch set
constexpr int kMaxBatch = 16;  // trajectories in one batched launch (etp_step_batch)
constexpr int kMaxBatchStep = 64;  // trajectories in one etp_step_batch call

struct Prm8 {
  double v[kMaxParams];
};

// --------------------------------------------------------------- profiling
enum KernelClass : int {
  KC_ELEM = 0, KC_GATHER = 1, KC_DOT = 2, KC_UPD_DOT = 3, KC_UPD_NORM = 4,
  KC_EXPM = 5, KC_COMBINE = 6, KC_OTHER = 7, KC_FUSED = 8, KC_FROZEN = 9, KC_LANCZOS = 10
};

struct ProfRecord {
  cudaEvent_t start, stop;
  int cls;
  double bytes;
  double flops;
};

}  // namespace etp

struct etp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  bool cooperative = false;  // device supports cooperative launches
  bool profiling = false;
  // switches read once from the environment when the context is created:
  // ETP_NO_PERSISTENT (separate-kernel Arnoldi steps for short vectors),
  // ETP_NO_COOP_EXPM (multi-launch a-priori checks), ETP_KRYLOV_WINDOW=W
  // (Arnoldi steps between checks, 1..8; 0 = built-in rule), ETP_NO_GRAPHS
  // (Newmark CG blocks launched directly instead of replayed graphs)
  bool no_persistent = false;
  bool no_fused = false;  // ETP_NO_FUSED_SOLVE: one launch per Arnoldi step even where the whole solve fits one
  bool no_coop_expm = false;
  int krylov_window = 0;
  bool no_graphs = false;
  // polls after which a grid-barrier wait of the persistent Arnoldi step gives
  // up (0 = built-in limit); lowered only by the test hook etp_debug_spin_limit
  unsigned long long pk_spin_limit = 0;
  std::vector<cudaEvent_t> event_pool;
  std::vector<etp::ProfRecord> records;
  int64_t prof_launches[ETP_NUM_KERNEL_CLASSES] = {};
  double prof_ms[ETP_NUM_KERNEL_CLASSES] = {};
  double prof_bytes[ETP_NUM_KERNEL_CLASSES] = {};
  double prof_flops[ETP_NUM_KERNEL_CLASSES] = {};
  std::atomic<int64_t> launches{0};  // host threads of a ragged batch may count at once
  // scratch for single-kernel entry points
  double* expm_ws = nullptr;
  size_t expm_ws_bytes = 0;
  // staging of the batched checks (batch_solve.cu): scaling exponents of all
  // candidates and copies of the checked solves' states, device and pinned host
  int* d_chk_s = nullptr;
  int* h_chk_s = nullptr;
  void* d_chk_ks = nullptr;
  void* h_chk_ks = nullptr;
};

// Mesh with constant data on the device. Node vectors use a padded
// structure-of-arrays layout: component c of node n lives at c*nn_pad + n.
struct etp_mesh {
  etp_ctx* ctx = nullptr;
  int order = 1;
  int nen = 8;  // nodes per element
  int nq = 8;   // Gauss points per element
  int64_t n_nodes = 0, n_elems = 0, nn_pad = 0;
  // box detection (uniform lexicographic box): constant geometry
  bool is_box = false;
  int box_n[3] = {0, 0, 0};
  double box_h[3] = {0, 0, 0};
  // host copies
  std::vector<double> h_coords;
  std::vector<int32_t> h_conn;
  std::vector<uint8_t> h_fixed;  // per node, bit c set if component c is fixed
  // device
  int32_t* d_conn = nullptr;     // n_elems*nen
  int32_t* d_inc_ptr = nullptr;  // node -> incident (element, local node) CSR
  int32_t* d_inc_idx = nullptr;  // entries e*nen + A, ascending
  uint8_t* d_fixed = nullptr;    // n_nodes
  double* d_geo64 = nullptr;     // general meshes: per (e,q): Jinv (9) + dV (1)
  double* d_qtab64 = nullptr;    // Q1: lane constants of the FP64 element pass (k_q1_lane_table)
  float* d_geo32 = nullptr;
  // reference tables (host-computed, copied per launch as kernel constants)
  double dN_ref[etp::kMaxQ][etp::kMaxNen][3];  // reference gradients at Gauss points
  double w_ref[etp::kMaxQ];               // Gauss weights (tensor product)
  double w_gll[etp::kMaxNen];             // GLL weights at the nodes
  // material
  bool material_ready = false;
  int material_version = 0;  // incremented by etp_material_set (invalidates stored frozen coefficients)
  int kind = 0;
  double params[etp::kMaxParams] = {};
  double rho = 1.0;
  float* d_escale = nullptr;       // n_elems or null
  double* d_msqrt = nullptr;       // per node sqrt(m)
  double* d_minvsqrt64 = nullptr;  // per node 1/sqrt(m)
  float* d_minvsqrt32 = nullptr;
  std::vector<double> h_mass;      // per node
};

namespace etp {

// Frozen-state description for one operator application.
struct FrozenSet {
  int count = 0;               // 0: u* = 0 (or linear), 1 or 2 states
  const void* u[2] = {nullptr, nullptr};  // SoA, 3*nn_pad, precision of the apply
  double c[2] = {1.0, 0.0};    // combination weights
  const void* data[2] = {nullptr, nullptr};  // stored frozen coefficients (build_frozen)
  int slot[2] = {-1, -1};      // midpoint-history slot of each state (its coefficients are kept), or -1
};

// Device-side status of a Krylov solve.
struct KState {
  int stop;        // 1: no further Arnoldi iterations (breakdown or converged)
  int breakdown_j; // Krylov size at which a happy breakdown occurred (0 = none)
  int err;         // KERR_*
  int found_m;     // selected Krylov size (0 = not yet)
  double eps;      // estimate of the selected size
  double beta;     // ||w||
  double hnorm2;   // running ||H_j||_F^2
  int converged;
  int pad;
};

}  // namespace etp

struct etp_traj {
  etp_mesh* mesh = nullptr;
  int prec = ETP_PREC_FP64;
  int m_cap = 0;
  int64_t L = 0;  // 6*nn_pad
  int64_t steps = 0;
  // state and buffers (FP64 unless noted)
  double* d_w = nullptr;       // state w_bar (L)
  double* d_wtmp = nullptr;    // predictor result / scratch (L)
  void* d_V = nullptr;         // basis (m_cap+1) x L, precision T
  void* d_z = nullptr;         // Arnoldi work vector (L), precision T
  void* d_Ye = nullptr;        // element contributions n_elems*nen*3, precision T
  void* d_hist[3] = {nullptr, nullptr, nullptr};  // frozen displacements, 3*nn_pad, T
  // stored frozen coefficients per midpoint-history slot (T): built when the
  // slot's state is first used as a frozen state, reused while it is unchanged
  void* d_fz[3] = {nullptr, nullptr, nullptr};
  bool fz_valid[3] = {false, false, false};
  int fz_version = -1;                 // material version the coefficients belong to
  size_t fz_bytes = 0;                 // bytes of each d_fz buffer
  size_t device_bytes = 0;             // device memory of this trajectory (traj_device_bytes)
  // constant external load (Section 2.3, augmented state [u_bar; v_bar; 1]):
  // P_bar = M^{-1/2} P per free DOF (SoA, 3*nn_pad) in the apply precision and
  // in FP64 (energy); the augmented entry is row 3*nn_pad - 1 of the state
  bool has_load = false;
  void* d_pbar = nullptr;
  double* d_pbar64 = nullptr;
  int hist_count = 0;          // midpoint states available (0, 1, 2)
  int hist_newest = 0;         // slot index of u_{n-3/2}
  double* d_H = nullptr;       // Hessenberg (m_cap+1) x m_cap column-major FP64
  double* d_coef = nullptr;    // per column: h1 (m_cap+1), h2, g (update coefs), colscale
  double* d_partials = nullptr;  // per-block partial sums
  unsigned int* d_counter = nullptr;  // last-block-done counters
  etp::KState* d_ks = nullptr;
  etp::KState* h_ks = nullptr;  // pinned mirror
  double* d_y = nullptr;       // beta * exp(tau H_m) e_1 (m_cap)
  double* d_expm_ws = nullptr; // small exponential workspace
  int expm_ws_cand = 0;        // candidates the workspace holds
  double* d_red = nullptr;     // scalar reductions scratch
  int last_m = 0;
  int m_hint[2] = {0, 0};
  int krylov = ETP_KRYLOV_ARNOLDI;  // etp_krylov_method
  // Newmark-beta path (newmark.cu): FP64 workspace allocated at its first step,
  // and whether the stored acceleration belongs to the current state
  void* d_nm = nullptr;
  bool nm_valid = false;
  void* nm_exec = nullptr;  // captured CG block (cudaGraphExec_t) and what it was captured for
  int nm_exec_kind = -1;
  double nm_exec_c = 0.0;      // Krylov size of the previous solve of each kind (0: corrector/linear, 1: predictor)
};
