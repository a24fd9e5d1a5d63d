// Persistent Arnoldi step for small vectors (Section 4.3): the node gather of
// z = A v_j and the three CGS2 passes in ONE cooperative launch, separated by
// barriers over the trajectory's blocks instead of kernel boundaries and
// last-block reductions. Each pass writes one partial sum per (column, tile);
// each coefficient reduction is spread over the blocks (block b sums column b
// over the tiles in a fixed order), followed by one barrier after which every
// block reads the coefficients. For vectors of up to a few hundred thousand
// rows the work per pass is a few microseconds, so launch and reduction
// latency, not bandwidth, set the step time; this kernel removes most of it.
// The batched form runs the steps of several trajectories in one launch.
#pragma once

#include "fe_kernels.cuh"
#include "krylov_kernels.cuh"

namespace etp {

// Polls of a waiting block before it gives up (each poll is an L2 round trip,
// ~0.3-1 us: the limit is several seconds, far beyond any legitimate wait).
constexpr unsigned long long kBarrierSpinLimit = 1ull << 23;

// Release / acquire operations at GPU scope (PTX memory model): lighter than a
// full fence, and enough to order a block's writes before a barrier arrival and
// the reads after it.
__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;\n" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned int* p, unsigned int v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Barrier over the nb blocks that work on one trajectory (all of a
// cooperative launch, or one trajectory's share of a batched launch; every
// block is co-resident). The block's writes are ordered before thread 0's
// arrival by __syncthreads and the release of the arrival; the last block
// to arrive acquires them all, resets the counter and releases the next
// generation; the others acquire it, and __syncthreads hands the view to the
// whole block. Bounded: a block that waits `limit` polls records KERR_TIMEOUT
// in *err and continues, so the kernel always ends; the host reports
// ETP_ERR_TIMEOUT and does not commit the step.
__device__ __forceinline__ void group_barrier(unsigned int* count, unsigned int* gen, int* err, int nb,
                                              unsigned long long limit = kBarrierSpinLimit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire_gpu(gen);  // generation before this block arrives
    if (atom_add_acq_rel_gpu(count, 1u) == (unsigned int)nb - 1) {
      st_relaxed_gpu(count, 0u);
      st_release_gpu(gen, g + 1u);
    } else {
      unsigned long long spins = 0;
      while (ld_acquire_gpu(gen) == g) {
        if (++spins > limit) {
          atomicOr(err, KERR_TIMEOUT);
          break;
        }
      }
    }
  }
  __syncthreads();
}

template <typename T>
struct PkParams {
  int64_t n_nodes, nn_pad;
  const int32_t* inc_ptr;
  const int32_t* inc_idx;
  const T* Ye;            // element contributions of A v_j
  const T* minvsqrt;
  const uint8_t* fixed;
  const T* xb;            // bottom half of v_j (stored column)
  const double* xscale;   // column scale of v_j
  CgsParams<T> c;         // basis, z, coefficients, partials, Hessenberg, state
  const T* pbar;          // loaded state: P_bar (SoA 3*nn_pad) and the augmented entry of v_j
  const T* xi;
  unsigned int* bar_count;
  unsigned int* bar_gen;
  // polls before a barrier wait gives up: kBarrierSpinLimit, or the lower
  // limit a test sets (etp_debug_spin_limit) to make the wait run out. Only
  // this kernel's barriers take it: every loop bound and index here is a
  // launch parameter, so a block that leaves a barrier early computes wrong
  // values but stays in bounds and ends.
  unsigned long long spin_limit;
};

// Doubles of partial sums one persistent step of j columns and TR-row tiles
// needs: two dot passes of j columns and one norm pass, one value per tile.
__host__ __device__ constexpr int64_t pk_partials_count(int64_t L, int j, int TR) {
  return (2 * (int64_t)j + 1) * (L / TR);
}

// Tile rows of the persistent step for j columns: the largest of 128, 64, 32
// whose two staged tiles fit 200 KB of shared memory.
constexpr size_t kPkSmemMax = 200 * 1024;
template <typename T>
constexpr int pk_tile_rows(int j) {
  return cgs_smem_bytes<T>(j, 128) <= kPkSmemMax ? 128 : cgs_smem_bytes<T>(j, 64) <= kPkSmemMax ? 64 : 32;
}

// Vectors of at most this many tiles reduce redundantly (every block sums every
// column itself: no barrier after the reduction).
constexpr int64_t kPkRedundantTiles = 64;

// Redundant reduction for few tiles: warp w sums columns w, w+4, ... over the
// tiles (lane k takes tiles k, k+32, ..., then a shuffle tree): every block
// gets the same values in the same order, independent of the block count;
// block 0 stores h_i and g_i.
template <typename T>
__device__ __forceinline__ void pk_reduce_redundant(const double* part, int64_t ntiles, int j, int bid,
                                                    const double* scale, double* coef_h, double* coef_g, T* s_g) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < j; i += nw) {
    double d = 0.0;
    for (int64_t t = lane; t < ntiles; t += 32) d += __ldcg(part + (int64_t)i * ntiles + t);
    d = warp_sum(d);
    const double h = scale[i] * d;
    if (lane == 0) {
      s_g[i] = (T)(scale[i] * h);
      if (bid == 0) {
        coef_h[i] = h;
        coef_g[i] = scale[i] * h;
      }
    }
  }
  __syncthreads();
}

// Distributed reduction: block b sums columns b, b+nb, ... over the tiles
// (thread k takes tiles k, k+128, ... in order, then a fixed tree), writes
// h_i and g_i; after a barrier every block reads the j update coefficients.
template <typename T>
__device__ __forceinline__ void pk_reduce_distributed(const double* part, int64_t ntiles, int j, int bid, int nb,
                                                      const double* scale, double* coef_h, double* coef_g,
                                                      double* s_red, T* s_g, unsigned int* bc, unsigned int* bg,
                                                      int* err, unsigned long long limit) {
  for (int i = bid; i < j; i += nb) {
    double d = 0.0;
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) d += __ldcg(part + (int64_t)i * ntiles + t);
    d = block_sum(d, s_red);
    if (threadIdx.x == 0) {
      const double h = scale[i] * d;
      coef_h[i] = h;
      coef_g[i] = scale[i] * h;
    }
  }
  group_barrier(bc, bg, err, nb, limit);
  for (int i = threadIdx.x; i < j; i += blockDim.x) s_g[i] = (T)__ldcg(coef_g + i);
  __syncthreads();
}

// One Arnoldi step of one trajectory on blocks bid = 0..nb-1 of its group.
template <typename T, int TR>
__device__ __forceinline__ void pk_step(const PkParams<T>& p, int bid, int nb, unsigned char* smem_raw) {
  KState* ks = p.c.ks;
  if (__ldcg(&ks->stop)) return;  // written before a barrier (or between launches): the same for every block
  constexpr int BD = 128;
  __shared__ T s_g[kMaxCap];
  __shared__ double s_red[32];
  __shared__ double s_tmp[BD];
  const int tid = threadIdx.x, j = p.c.j;
  const int64_t ntiles = p.c.L / TR;
  int* err = &ks->err;
  double* coef = p.c.coef;
  const double* scale = coef + COEF_SCALE * COEF_STRIDE;
  TilePartials pt1{p.c.partials, nullptr};
  TilePartials pt2{p.c.partials + (int64_t)j * ntiles, nullptr};
  TilePartials ptn{nullptr, p.c.partials + 2 * (int64_t)j * ntiles};

  // ---- phase A: z = A v_j (node gather of the element terms, top half copy)
  {
    const int64_t nn = p.nn_pad;
    T* zt = p.c.z;
    T* zb = p.c.z + 3 * nn;
    const T xs = (T)(*p.xscale);
    const T lx = p.pbar ? (*p.xi) * xs : T(0);
    for (int64_t n = (int64_t)bid * BD + tid; n < nn; n += (int64_t)nb * BD) {
      if (n >= p.n_nodes) {
#pragma unroll
        for (int c = 0; c < 3; ++c) { zt[c * nn + n] = T(0); zb[c * nn + n] = T(0); }
        continue;
      }
      T a0 = T(0), a1 = T(0), a2 = T(0);
      for (int k = p.inc_ptr[n]; k < p.inc_ptr[n + 1]; ++k) {
        const T* y = p.Ye + (int64_t)p.inc_idx[k] * 3;
        a0 += y[0]; a1 += y[1]; a2 += y[2];
      }
      T l0 = T(0), l1 = T(0), l2 = T(0);
      if (p.pbar) { l0 = lx * p.pbar[n]; l1 = lx * p.pbar[nn + n]; l2 = lx * p.pbar[2 * nn + n]; }
      const T s = -p.minvsqrt[n];
      const uint8_t f = p.fixed[n];
      zb[n] = (f & 1) ? T(0) : s * a0 + l0;
      zb[nn + n] = (f & 2) ? T(0) : s * a1 + l1;
      zb[2 * nn + n] = (f & 4) ? T(0) : s * a2 + l2;
#pragma unroll
      for (int c = 0; c < 3; ++c) zt[c * nn + n] = p.xb[c * nn + n] * xs;
    }
  }
  group_barrier(p.bar_count, p.bar_gen, err, nb, p.spin_limit);

  // ---- phase B: h1 = V^T z
  const bool redundant = ntiles <= kPkRedundantTiles;
  cgs_tiles<T, CGS_DOT, TR>(p.c, smem_raw, s_g, bid, nb, pt1, s_tmp, s_red);
  group_barrier(p.bar_count, p.bar_gen, err, nb, p.spin_limit);
  if (redundant)
    pk_reduce_redundant<T>(pt1.dots, ntiles, j, bid, scale, coef + COEF_H1 * COEF_STRIDE, coef + COEF_G * COEF_STRIDE,
                           s_g);
  else
    pk_reduce_distributed<T>(pt1.dots, ntiles, j, bid, nb, scale, coef + COEF_H1 * COEF_STRIDE,
                             coef + COEF_G * COEF_STRIDE, s_red, s_g, p.bar_count, p.bar_gen, err, p.spin_limit);

  // ---- phase C: z -= V g1, h2 = V^T z
  cgs_tiles<T, CGS_UPD_DOT, TR>(p.c, smem_raw, s_g, bid, nb, pt2, s_tmp, s_red);
  group_barrier(p.bar_count, p.bar_gen, err, nb, p.spin_limit);
  if (redundant)
    pk_reduce_redundant<T>(pt2.dots, ntiles, j, bid, scale, coef + COEF_H2 * COEF_STRIDE, coef + COEF_G * COEF_STRIDE,
                           s_g);
  else
    pk_reduce_distributed<T>(pt2.dots, ntiles, j, bid, nb, scale, coef + COEF_H2 * COEF_STRIDE,
                             coef + COEF_G * COEF_STRIDE, s_red, s_g, p.bar_count, p.bar_gen, err, p.spin_limit);

  // ---- phase D: z -= V g2 -> new basis column, ||z||^2 per tile
  cgs_tiles<T, CGS_UPD_NORM, TR>(p.c, smem_raw, s_g, bid, nb, ptn, s_tmp, s_red);
  group_barrier(p.bar_count, p.bar_gen, err, nb, p.spin_limit);
  if (bid != 0) return;
  // ---- block 0: Hessenberg column, breakdown test, scale of the new column
  double n2 = 0.0;
  for (int64_t t = tid; t < ntiles; t += BD) n2 += __ldcg(ptn.norm + t);
  n2 = block_sum(n2, s_red);
  const int col = j - 1;
  double hsq = 0.0;
  for (int i = tid; i < j; i += BD) {
    const double h = coef[COEF_H1 * COEF_STRIDE + i] + coef[COEF_H2 * COEF_STRIDE + i];
    p.c.H[i + (int64_t)col * p.c.ldH] = h;
    hsq += h * h;
  }
  const double colsum = block_sum(hsq, s_red);
  if (tid == 0) {
    const double hn2 = ks->hnorm2 + colsum;
    const double hn = sqrt(n2);
    p.c.H[j + (int64_t)col * p.c.ldH] = hn;
    if (!isfinite(hn) || !isfinite(hn2)) {
      ks->err |= KERR_NONFINITE;
      ks->stop = 1;
    } else if (hn <= 1e-14 * sqrt(hn2)) {
      ks->breakdown_j = j;
      ks->stop = 1;
    } else {
      coef[COEF_SCALE * COEF_STRIDE + j] = 1.0 / hn;
    }
    ks->hnorm2 = hn2 + hn * hn;
    if (ks->err & KERR_TIMEOUT) ks->stop = 1;
  }
}

template <typename T, int TR>
static __global__ void __launch_bounds__(128) k_arnoldi_step_pk(PkParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pk_step<T, TR>(p, blockIdx.x, gridDim.x, smem_raw);
}

// Ragged batch: the Arnoldi steps of up to kMaxBatch trajectories (each its
// own mesh, size and column count j, one tile size) in one cooperative launch.
// Trajectory i owns blocks off[i] .. off[i+1]-1 and synchronises only them.
template <typename T>
struct PkBatch {
  int n;
  int off[kMaxBatch + 1];
  PkParams<T> item[kMaxBatch];
};

template <typename T, int TR>
static __global__ void __launch_bounds__(128) k_arnoldi_step_pk_batch(const __grid_constant__ PkBatch<T> b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int i = 0;
  while (i + 1 < b.n && (int)blockIdx.x >= b.off[i + 1]) ++i;
  pk_step<T, TR>(b.item[i], (int)blockIdx.x - b.off[i], b.off[i + 1] - b.off[i], smem_raw);
}

}  // namespace etp
