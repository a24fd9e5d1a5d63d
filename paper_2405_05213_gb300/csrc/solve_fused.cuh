// A whole Krylov solve of one trajectory with short vectors in ONE cooperative
// launch (Section 4.3): for j = 1, 2, ... the element pass of column j-1, the
// persistent Arnoldi step (node gather and the CGS2 passes), and at the check
// points the a-priori estimate (Eq. "subspace error estimate") for every size
// of the window, with the selection of the smallest passing size made on the
// device; the loop stops there. The host synchronises once per solve instead
// of once per check window, and no launch gap separates the steps.
//
// Every value is computed by the same device functions and in the same order
// as in the separate launches (element pass: per element; Arnoldi step: per
// tile, in tile order, with the tile size of its column count; checks: per
// candidate and entry), so the result is bit for bit that of the launch-per-
// step path. All waits are the bounded grid barriers of the persistent step.
//
// Blocks read, after a barrier, data other blocks wrote earlier in the same
// launch (basis columns, element terms, Hessenberg entries, scales). The grid
// barrier's arrival is a release and its wait an acquire at GPU scope, so under
// the PTX memory model every read after it (plain loads and the Gram-Schmidt
// tiles' copies alike) observes those writes, as within the persistent step.
#pragma once

#include "arnoldi_pk.cuh"
#include "expm_kernels.cuh"

namespace etp {

// Scaling, Paterson-Stockmeyer products and squarings of the candidates of one
// check on blocks bid = 0..nb-1 (the stages of the single-launch check; the
// number of squarings is read from the scaling exponents on the device).
__device__ __forceinline__ void expm_window_stages(const ExpmParams& p, int bid, int nb, GridBar& gb) {
  for (int c = bid; c < p.ncand; c += nb) {
    expm_prep_cand(p, c);
    __syncthreads();
  }
  gb.sync();
  const int jmax = p.j0 + p.ncand - 1;
  const int per = jmax * jmax;
  const int64_t total = (int64_t)per * p.ncand;
  auto stage = [&](int st, int k, int z) {
    for (int64_t w = (int64_t)bid * blockDim.x + threadIdx.x; w < total; w += (int64_t)nb * blockDim.x)
      expm_mm_entry(p, (int)(w / per), (int)(w % per), z, st, k);
  };
  stage(0, 0, 0);
  gb.sync();
  stage(1, 0, 0);
  stage(1, 0, 1);
  gb.sync();
  for (int k = 3; k >= 0; --k) {
    stage(2, k, 0);
    gb.sync();
  }
  // s <= 1024 for every finite |tau H| (the exponent range of a double): the
  // clamp only bounds the loop should a stale exponent ever be read
  int smax = 0;
  for (int c = 0; c < p.ncand; ++c) smax = max(smax, __ldcg(p.s_arr + c));
  smax = min(smax, 1024);
  for (int k = 0; k < smax; ++k) {
    stage(3, k, 0);
    gb.sync();
  }
}

template <typename T>
struct FusedSolve {
  ApplyParams<T> ap;  // element pass (x and xscale set per step)
  PkParams<T> pk;     // persistent step (column fields set per step)
  ExpmParams ex;      // checks (j0 and ncand set per window)
  KState* ks;
  T* V;
  const double* scale;  // coef + COEF_SCALE * COEF_STRIDE
  int j_end;            // last Arnoldi step of this launch (<= cap)
  int cap;              // the solve's capacity (m_fixed or m_cap)
  int first_check, W, m_fixed;
  double tol;
  double* e_out;
};

template <typename T>
__device__ __forceinline__ void fused_pk_step(const PkParams<T>& q, int tr, int bid, int nb, unsigned char* smem,
                                              GridBar& gb) {
  switch (tr) {
    case 256: pk_step<T, 256>(q, bid, nb, smem, gb); break;
    case 128: pk_step<T, 128>(q, bid, nb, smem, gb); break;
    case 64: pk_step<T, 64>(q, bid, nb, smem, gb); break;
    default: pk_step<T, 32>(q, bid, nb, smem, gb); break;
  }
}

template <typename T, int KIND, int NS>
static __global__ void __launch_bounds__(128) k_krylov_solve_fused(const __grid_constant__ FusedSolve<T> f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = gridDim.x, bid = blockIdx.x;
  KState* ks = f.ks;
  const int64_t L = f.pk.c.L, nn = f.pk.nn_pad;
  GridBar gb = make_grid_bar(f.pk.bar, &ks->err, nb, f.pk.spin_limit);
  int win_start = 1;
  int next_check = f.first_check;
  int res_tr = 0;  // tile rows of the last step, while this block keeps its tile in shared memory
  for (int j = 1; j <= f.j_end; ++j) {
    const T* x = f.V + (int64_t)(j - 1) * L;
    ApplyParams<T> a = f.ap;
    a.x = x;
    a.xscale = f.scale + (j - 1);
    elem_apply_blocks<1, T, KIND, true, NS>(a, bid, nb);
    gb.sync();
    PkParams<T> q = f.pk;
    q.c.j = j;
    q.c.vout = f.V + (int64_t)j * L;
    q.xb = x + 3 * nn;
    q.xscale = f.scale + (j - 1);
    q.xi = q.pbar ? x + 3 * nn - 1 : nullptr;
    // one tile per block: columns 0..j-1 of the tile are still in shared memory
    // if the last step had the same tile rows (its z'' is column j-1)
    const int tr = pk_tile_rows<T>(j, L);
    const bool single = pk_ntiles(L, tr) <= nb;
    q.res_cols = (single && tr == res_tr) ? j : 0;
    fused_pk_step<T>(q, tr, bid, nb, smem_raw, gb);
    res_tr = single ? tr : 0;
    gb.sync();  // column j of H, its scale and the stop flag are visible
    if (j != next_check) continue;
    int lo = win_start, hi = j, target = 0;
    if (f.m_fixed > 0) {
      const int jb = __ldcg(&ks->breakdown_j);
      lo = hi = target = (jb > 0 ? jb : f.cap);
      if (__ldcg(&ks->beta) == 0.0) lo = hi = target = 1;
    }
    bool done = __ldcg(&ks->err) != 0;
    for (int j0 = lo; j0 <= hi && !done; j0 += kMaxCand) {
      ExpmParams e = f.ex;
      e.j0 = j0;
      e.ncand = min(hi, j0 + kMaxCand - 1) - j0 + 1;
      expm_window_stages(e, bid, nb, gb);
      if (bid == 0) expm_select_block(e, ks, f.tol, target, (j0 + e.ncand - 1 >= f.cap) ? 1 : 0, f.e_out);
      gb.sync();
      done = __ldcg(&ks->err) != 0 || __ldcg(&ks->found_m) >= 0;
    }
    if (done) break;
    win_start = j + 1;
    next_check = min(f.j_end, j + f.W);
  }
}

}  // namespace etp
