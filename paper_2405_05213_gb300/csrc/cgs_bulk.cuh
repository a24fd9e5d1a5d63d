// Gram-Schmidt passes over long vectors with bulk asynchronous copies
// (Section 4.3, orthogonalisation of the Arnoldi vectors: classical
// Gram-Schmidt with one reorthogonalisation, organised in two passes per step
// as described at BulkMode below).
//
// The rows are cut into tiles of TR rows. For each tile the lanes of warp 0
// issue one 1-D bulk copy (cp.async.bulk, the TMA engine's linear mode) per
// basis column and one for z into a shared-memory stage; the copies complete
// on the stage's mbarrier. A stage is refilled as soon as its tile has been
// used, so up to NS tiles per block are in flight while the block waits and
// NS - 1 while it computes.
//
// Work split inside a tile (256 threads = 8 warps, vectors of VEC = 16 /
// sizeof(T) elements):
//  * updates (BULK_UPD: the new q_j and the next candidate, two linear
//    combinations of the same staged columns): thread t owns vectors of rows;
//    for short tiles the columns are split over G thread groups and combined
//    in a fixed order through shared memory.
//  * dots    h_i = V_i . x (x = z, or the new candidate): warp w takes
//    columns w, w+8, ...; its lanes stride over the tile's vectors (16-byte
//    shared loads, no bank conflicts) and keep one running sum per column
//    across all of the block's tiles.
//
// Accumulation in MIXED precision. FP64 arithmetic is a small fraction of the
// FP32 rate on this GPU, so the running sums are float-float pairs (hi, lo)
// updated with Knuth's TwoSum (error-free addition, 6 FP32 operations): a
// lane's products of one tile (at most 16 per chain) are summed in FP32 and
// the tile value enters the pair without rounding error. The pairs are
// reduced across lanes and blocks in float-float as well (block partials are
// stored as (hi, lo) in the 8-byte partial slots) and turned into a double
// once per column. In FP64 precision everything is plain double.
//
// Every wait on an mbarrier is bounded; a block that gives up records
// KERR_TIMEOUT, waits (bounded) for its copies still in flight and takes part
// in the last-block reduction so the launch always ends cleanly.
#pragma once

#include "krylov_kernels.cuh"

namespace etp {

constexpr int kBulkMaxStages = 4;
constexpr int kBulkWaitLimit = 1 << 22;  // try_wait polls before a block gives up (seconds)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      " .reg .pred P;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
      " selp.u32 %0, 1, 0, P;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier to complete, at most kBulkWaitLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (int it = 0; it < kBulkWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Linear global -> shared copy of `bytes` (multiple of 16, both ends 16-byte
// aligned) that signals the barrier's transaction count when it lands.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <typename T>
struct BulkVec;
template <>
struct BulkVec<float> {
  using V = float4;
  static constexpr int N = 4;
  __device__ static __forceinline__ float dot(const float4 a, const float4 b, float acc) {
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
  }
  __device__ static __forceinline__ float4 axpy(float g, const float4 a, float4 y) {
    return make_float4(fmaf(g, a.x, y.x), fmaf(g, a.y, y.y), fmaf(g, a.z, y.z), fmaf(g, a.w, y.w));
  }
  __device__ static __forceinline__ float4 sub(const float4 a, const float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
  }
  __device__ static __forceinline__ float4 add(const float4 a, const float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
  }
  __device__ static __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static __forceinline__ float sumsq(const float4 a) {
    return fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, a.w * a.w)));
  }
};
template <>
struct BulkVec<double> {
  using V = double2;
  static constexpr int N = 2;
  __device__ static __forceinline__ double dot(const double2 a, const double2 b, double acc) {
    acc = fma(a.x, b.x, acc);
    return fma(a.y, b.y, acc);
  }
  __device__ static __forceinline__ double2 axpy(double g, const double2 a, double2 y) {
    return make_double2(fma(g, a.x, y.x), fma(g, a.y, y.y));
  }
  __device__ static __forceinline__ double2 sub(const double2 a, const double2 b) {
    return make_double2(a.x - b.x, a.y - b.y);
  }
  __device__ static __forceinline__ double2 add(const double2 a, const double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
  }
  __device__ static __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  __device__ static __forceinline__ double sumsq(const double2 a) { return fma(a.x, a.x, a.y * a.y); }
};

template <typename T>
__device__ __forceinline__ T warp_allsum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kBulkThreads = 256;

// The two passes of one Arnoldi step on long vectors (CGS2 with the second
// pass of column j carried out together with the first pass of column j+1).
//
// State at step j: q_1..q_{j-1} are final (stored columns 0..j-2 with their
// scales), column j-1 holds the candidate u_j (u_j = s_u V_{j-1}, projected
// once), together with its reorthogonalisation coefficients a = Q^T u_j and
// r = ||u_j - Q a|| (from the previous step). z = A u_j.
//  BULK_DOT: b = Q^T z, gamma = u_j^T z (one read of the j columns and z);
//    then, in the last block, the small algebra: q_j^T z = (gamma - a.b)/r and,
//    through the Arnoldi relation A Q = Q_j H, the first-pass coefficients of
//    A q_j, h1 = (Q_j^T z - H a)/r, and the update coefficients of
//    u_{j+1} = (z - Q_j Q_j^T z)/r = (z - c u_j - Q (b - c a))/r, c = (gamma - a.b)/r^2.
//  BULK_UPD: per row, q_j = (u_j - Q a)/r (written over column j-1) and
//    r u_{j+1} (written to column j), from the same staged tile; then the dots of
//    the new candidate with Q_j, and its squared norm (an extra partial column),
//    give its coefficients a' and norm,
//    hence h_{1:j,j} = h1 + a' and h_{j+1,j} = r' = sqrt(|u_{j+1}|^2 - |a'|^2).
// In exact arithmetic this is classical Gram-Schmidt with one
// reorthogonalisation (the Hessenberg matrix and basis are those of CGS2); the
// basis is read twice per step instead of three times.
enum BulkMode : int { BULK_DOT = 0, BULK_UPD = 1 };

// Dynamic shared memory of k_cgs_bulk: NS stages of (j + 1) x TR elements,
// the new candidate tile, and the partial updates of the column groups (two
// sets in BULK_UPD).
template <typename T>
__host__ __device__ constexpr size_t cgs_bulk_smem_bytes(int j, int TR, int NS, int mode) {
  return (size_t)NS * (j + 1) * TR * sizeof(T) + (size_t)TR * sizeof(T) +
         (size_t)kBulkThreads * 16 * (mode == BULK_UPD ? 2 : 1);
}

// Raw column sums t_i (i < ncols) of the block partials, in a fixed order
// (deterministic for a fixed grid), into out[i]. `scratch` holds kBulkThreads
// 16-byte entries.
template <typename T>
__device__ __forceinline__ void reduce_columns(const CgsParams<T>& p, int ncols, double* out, unsigned char* scratch) {
  constexpr int BD = kBulkThreads;
  const int tid = threadIdx.x;
  const int nb = gridDim.x;
  T* s_pair = reinterpret_cast<T*>(scratch);  // [2 * BD]
  const int jc = ncols < BD ? ncols : BD;
  const int S = BD / jc;
  for (int i0 = 0; i0 < ncols; i0 += jc) {
    const int col = i0 + tid % jc, sub = tid / jc;
    T hi = T(0), lo = T(0);
    if (sub < S && col < ncols) {
      const double* pc = p.partials + (int64_t)col * nb;
      for (int b = sub; b < nb; b += S) {
        T h2, l2;
        load_partial(pc + b, h2, l2);
        acc_add_pair(hi, lo, h2, l2);
      }
    }
    __syncthreads();
    if (sub < S) {
      s_pair[2 * (sub * jc + tid % jc)] = hi;
      s_pair[2 * (sub * jc + tid % jc) + 1] = lo;
    }
    __syncthreads();
    if (tid < jc && i0 + tid < ncols) {
      T h = s_pair[2 * tid], l = s_pair[2 * tid + 1];
      for (int k = 1; k < S; ++k) acc_add_pair(h, l, s_pair[2 * (k * jc + tid)], s_pair[2 * (k * jc + tid) + 1]);
      out[i0 + tid] = pair_value(h, l);
    }
  }
  __syncthreads();
}

// Last block of BULK_DOT: b, gamma -> h1 and the coefficients of BULK_UPD.
template <typename T>
__device__ __forceinline__ void bulk_dot_finalize(const CgsParams<T>& p, unsigned char* scratch, double* s_red) {
  constexpr int BD = kBulkThreads;
  const int j = p.j, tid = threadIdx.x;
  double* coef = p.coef;
  const double* scale = coef + COEF_SCALE * COEF_STRIDE;
  double* bz = coef + COEF_H1 * COEF_STRIDE;  // b_i (i < j-1), gamma (i = j-1)
  reduce_columns(p, j, bz, scratch);
  for (int i = tid; i < j; i += BD) bz[i] *= scale[i];
  __syncthreads();
  const double* a = coef + COEF_A * COEF_STRIDE;
  double* misc = coef + COEF_MISC * COEF_STRIDE;
  const double r = misc[MISC_R];
  const double su = scale[j - 1];
  double ab = 0.0;
  for (int i = tid; i < j - 1; i += BD) ab += a[i] * bz[i];
  ab = block_sum(ab, s_red);
  __shared__ double s_c;
  if (tid == 0) s_c = (bz[j - 1] - ab) / (r * r);
  __syncthreads();
  const double c = s_c;
  for (int i = tid; i < j - 1; i += BD) {
    coef[COEF_G * COEF_STRIDE + i] = a[i] * scale[i];
    coef[COEF_D * COEF_STRIDE + i] = (bz[i] - c * a[i]) * scale[i];
  }
  // h1_i = ((Q_j^T z)_i - (H a)_i) / r over the final columns 0..j-2 of H
  for (int i = tid; i < j; i += BD) {
    const double qz = (i < j - 1) ? bz[i] : c * r;
    double ha = 0.0;
    for (int k = 0; k < j - 1; ++k) ha += p.H[i + (int64_t)k * p.ldH] * a[k];
    coef[COEF_HT * COEF_STRIDE + i] = (qz - ha) / r;
  }
  if (tid == 0) {
    misc[MISC_SU] = su;
    misc[MISC_EU] = c * su;
    *p.counter = 0u;
  }
}

// Last block of BULK_UPD: a', r' -> Hessenberg column j-1, scales, breakdown.
template <typename T>
__device__ __forceinline__ void bulk_upd_finalize(const CgsParams<T>& p, unsigned char* scratch, double* s_red) {
  constexpr int BD = kBulkThreads;
  const int j = p.j, tid = threadIdx.x;
  double* coef = p.coef;
  double* scale = coef + COEF_SCALE * COEF_STRIDE;
  double* t = coef + COEF_H2 * COEF_STRIDE;  // raw dots with columns 0..j-1 and the candidate itself
  reduce_columns(p, j + 1, t, scratch);
  double* misc = coef + COEF_MISC * COEF_STRIDE;
  const double inv = 1.0 / misc[MISC_R];
  double* a = coef + COEF_A * COEF_STRIDE;
  const int col = j - 1;
  double aa = 0.0, hsq = 0.0;
  for (int i = tid; i < j; i += BD) {
    const double ai = (i < j - 1) ? scale[i] * t[i] * inv : t[i] * inv * inv;
    a[i] = ai;
    const double h = coef[COEF_HT * COEF_STRIDE + i] + ai;
    p.H[i + (int64_t)col * p.ldH] = h;
    aa += ai * ai;
    hsq += h * h;
  }
  aa = block_sum(aa, s_red);
  hsq = block_sum(hsq, s_red);
  if (tid == 0) {
    KState* ks = p.ks;
    const double alpha = t[j] * inv * inv;
    const double rn = sqrt(fmax(alpha - aa, 0.0));
    const double hn2 = ks->hnorm2 + hsq;
    p.H[j + (int64_t)col * p.ldH] = rn;
    scale[j - 1] = inv;  // q_j = V_{j-1} / r
    scale[j] = inv;      // u_{j+1} = V_j / r
    misc[MISC_R] = rn;
    if (!isfinite(rn) || !isfinite(hn2)) {
      ks->err |= KERR_NONFINITE;
      ks->stop = 1;
    } else if (rn <= 1e-14 * sqrt(hn2)) {
      ks->breakdown_j = j;
      ks->stop = 1;
    }
    ks->hnorm2 = hn2 + rn * rn;
    *p.counter = 0u;
  }
}

// One pass (MODE) over the rows; KA = column slots per warp (j <= 8 KA).
template <typename T, int MODE, int KA>
static __global__ void __launch_bounds__(kBulkThreads, 2) k_cgs_bulk(CgsParams<T> p, int TR, int NS) {
  using BV = BulkVec<T>;
  using VecT = typename BV::V;
  constexpr int VEC = BV::N;
  constexpr int BD = kBulkThreads;
  constexpr int NW = BD / 32;
  extern __shared__ __align__(128) unsigned char smem_bulk[];
  __shared__ T s_g[MODE == BULK_UPD ? kMaxCap : 1];
  __shared__ T s_d[MODE == BULK_UPD ? kMaxCap : 1];
  __shared__ double s_red[32];
  __shared__ __align__(8) uint64_t s_bar[kBulkMaxStages];
  if (p.ks->stop) return;
  const int j = p.j;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t L = p.L;
  const int64_t ntiles = (L + TR - 1) / TR;
  const size_t stage_elems = (size_t)(j + 1) * TR;
  T* const stages = reinterpret_cast<T*>(smem_bulk);
  T* const s_zn = stages + (size_t)NS * stage_elems;  // new candidate tile (BULK_UPD)
  VecT* const s_pu = reinterpret_cast<VecT*>(s_zn + TR);
  VecT* const s_pd = s_pu + BD;
  const int NVT = TR / VEC;                 // vectors in a full tile
  const int G = NVT >= BD ? 1 : BD / NVT;   // column groups of the update
  const int64_t nk = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  T* const Vq = p.V + (int64_t)(j - 1) * L;  // candidate column, overwritten by q_j
  T su = T(0), eu = T(0);

  if (MODE == BULK_UPD) {
    for (int i = tid; i < j - 1; i += BD) {
      s_g[i] = (T)p.coef[COEF_G * COEF_STRIDE + i];
      s_d[i] = (T)p.coef[COEF_D * COEF_STRIDE + i];
    }
    su = (T)p.coef[COEF_MISC * COEF_STRIDE + MISC_SU];
    eu = (T)p.coef[COEF_MISC * COEF_STRIDE + MISC_EU];
  }
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&s_bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  // warp 0 issues a tile: lane 0 arms the stage's barrier with the tile's
  // bytes, then the lanes issue the j + 1 copies in parallel
  auto issue = [&](int64_t k) {  // warp 0 only
    const int s = (int)(k % NS);
    const int64_t r0 = ((int64_t)blockIdx.x + k * gridDim.x) * TR;
    const int rows = (int)(L - r0 < (int64_t)TR ? L - r0 : (int64_t)TR);
    const unsigned bytes = (unsigned)rows * sizeof(T);
    T* dst = stages + (size_t)s * stage_elems;
    if (lane == 0) {
      // this stage was last written by the threads (BULK_UPD): order those
      // writes before the copy engine's
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive_expect_tx(&s_bar[s], bytes * (unsigned)(j + 1));
    }
    __syncwarp();
    for (int i = lane; i <= j; i += 32)
      bulk_copy_g2s(dst + (size_t)i * TR, (i < j ? p.V + (int64_t)i * L : p.z) + r0, bytes, &s_bar[s]);
  };
  int64_t k_issued = 0;  // warp 0: tiles issued so far
  if (warp == 0)
    for (; k_issued < nk && k_issued < NS; ++k_issued) issue(k_issued);

  T hi[KA], lo[KA];  // dots: column warp + NW * ka of this lane's vectors
#pragma unroll
  for (int ka = 0; ka < KA; ++ka) hi[ka] = lo[ka] = T(0);
  T nhi = T(0), nlo = T(0);  // BULK_UPD: squared norm of this thread's rows of the new candidate
  bool timed_out = false;
  int64_t k_fail = 0;  // first tile not consumed when a wait gave up
  for (int64_t k = 0; k < nk; ++k) {
    const int s = (int)(k % NS);
    const bool ok = mbar_wait_bounded(&s_bar[s], (unsigned)((k / NS) & 1));
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      k_fail = k;
      break;
    }
    const int64_t r0 = ((int64_t)blockIdx.x + k * gridDim.x) * TR;
    const int rows = (int)(L - r0 < (int64_t)TR ? L - r0 : (int64_t)TR);
    const int nv = rows / VEC;
    T* const Vt = stages + (size_t)s * stage_elems;
    VecT* const uv = reinterpret_cast<VecT*>(Vt + (size_t)(j - 1) * TR);  // candidate, then q_j
    const VecT* const zv = reinterpret_cast<const VecT*>(Vt + (size_t)j * TR);

    if (MODE == BULK_UPD) {
      // ---- q_j and the new candidate from the same rows:
      //   nq = s_u u - sum_i g_i V_i,  nu = z - e_u u - sum_i d_i V_i
      auto finish_row = [&](int v, VecT uq, VecT ud) {
        const VecT u = uv[v];
        const VecT nq = BV::sub(BV::axpy(su, u, BV::zero()), uq);
        const VecT nu = BV::sub(BV::sub(zv[v], BV::axpy(eu, u, BV::zero())), ud);
        reinterpret_cast<VecT*>(Vq + r0)[v] = nq;
        reinterpret_cast<VecT*>(p.vout + r0)[v] = nu;
        uv[v] = nq;
        reinterpret_cast<VecT*>(s_zn)[v] = nu;
        acc_add(nhi, nlo, BV::sumsq(nu));
      };
      if (G == 1) {
        for (int v = tid; v < nv; v += BD) {
          VecT uq = BV::zero(), ud = BV::zero();
#pragma unroll 4
          for (int i = 0; i < j - 1; ++i) {
            const VecT x = reinterpret_cast<const VecT*>(Vt + (size_t)i * TR)[v];
            uq = BV::axpy(s_g[i], x, uq);
            ud = BV::axpy(s_d[i], x, ud);
          }
          finish_row(v, uq, ud);
        }
      } else {
        const int v = tid % NVT, g = tid / NVT;
        if (v < nv) {
          VecT uq = BV::zero(), ud = BV::zero();
#pragma unroll 4
          for (int i = g; i < j - 1; i += G) {
            const VecT x = reinterpret_cast<const VecT*>(Vt + (size_t)i * TR)[v];
            uq = BV::axpy(s_g[i], x, uq);
            ud = BV::axpy(s_d[i], x, ud);
          }
          s_pu[g * NVT + v] = uq;
          s_pd[g * NVT + v] = ud;
        }
        __syncthreads();
        if (g == 0 && v < nv) {
          VecT uq = s_pu[v], ud = s_pd[v];
          for (int gg = 1; gg < G; ++gg) {
            uq = BV::add(uq, s_pu[gg * NVT + v]);
            ud = BV::add(ud, s_pd[gg * NVT + v]);
          }
          finish_row(v, uq, ud);
        }
      }
      __syncthreads();  // q_j and the candidate tiles complete before the dots
    }

    // ---- dots of columns 0..j-1 with the new candidate (BULK_UPD) or with z
    {
      const VecT* const zsrc = (MODE == BULK_DOT) ? zv : reinterpret_cast<const VecT*>(s_zn);
#pragma unroll
      for (int ka = 0; ka < KA; ka += 2) {
        const int ia = warp + NW * ka, ib = ia + NW;
        if (ia < j) {
          const bool two = ib < j;
          const VecT* const va = reinterpret_cast<const VecT*>(Vt + (size_t)ia * TR);
          const VecT* const vb = reinterpret_cast<const VecT*>(Vt + (size_t)(two ? ib : ia) * TR);
          T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0);
          int v = lane;
          for (; v + 32 < nv; v += 64) {
            const VecT z0 = zsrc[v], z1 = zsrc[v + 32];
            a0 = BV::dot(va[v], z0, a0);
            a1 = BV::dot(va[v + 32], z1, a1);
            if (two) {
              b0 = BV::dot(vb[v], z0, b0);
              b1 = BV::dot(vb[v + 32], z1, b1);
            }
          }
          if (v < nv) {
            const VecT z0 = zsrc[v];
            a0 = BV::dot(va[v], z0, a0);
            if (two) b0 = BV::dot(vb[v], z0, b0);
          }
          acc_add(hi[ka], lo[ka], a0 + a1);
          if (two) acc_add(hi[ka + 1], lo[ka + 1], b0 + b1);
        }
      }
    }
    // every thread is done with this stage: refill it with tile k + NS
    __syncthreads();
    if (warp == 0 && k_issued < nk) issue(k_issued++);
  }
  if (timed_out) {
    if (tid == 0) {
      atomicOr(&p.ks->err, (int)KERR_TIMEOUT);
      p.ks->stop = 1;
      // copies still in flight land in this block's shared memory: wait for them (bounded)
      for (int64_t k = k_fail; k < k_issued; ++k) mbar_wait_bounded(&s_bar[k % NS], (unsigned)((k / NS) & 1));
    }
    __syncthreads();
  }
  // ---- per-block partials, column-major: column i of block b at i * gridDim.x + b;
  // BULK_UPD adds the squared norm as column j
  if (MODE == BULK_UPD) {
    warp_allsum_pair(nhi, nlo);
    T* s_pair = reinterpret_cast<T*>(s_pu);
    __syncthreads();  // s_pu is free (the tile loop ended with a barrier)
    if (lane == 0) {
      s_pair[2 * warp] = nhi;
      s_pair[2 * warp + 1] = nlo;
    }
    __syncthreads();
    if (tid == 0) {
      T h = s_pair[0], l = s_pair[1];
      for (int w = 1; w < NW; ++w) acc_add_pair(h, l, s_pair[2 * w], s_pair[2 * w + 1]);
      store_partial(p.partials + (int64_t)j * gridDim.x + blockIdx.x, h, l);
    }
  }
#pragma unroll
  for (int ka = 0; ka < KA; ++ka) {
    const int i = warp + NW * ka;
    if (i < j) {
      T h = hi[ka], l = lo[ka];
      warp_allsum_pair(h, l);
      if (lane == 0) store_partial(p.partials + (int64_t)i * gridDim.x + blockIdx.x, h, l);
    }
  }
  if (!elect_last_block(p.counter)) return;
  if (MODE == BULK_DOT) bulk_dot_finalize<T>(p, smem_bulk, s_red);
  else bulk_upd_finalize<T>(p, smem_bulk, s_red);
}

}  // namespace etp
