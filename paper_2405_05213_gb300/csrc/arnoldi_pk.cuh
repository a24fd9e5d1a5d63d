// Persistent Arnoldi step for short vectors (Section 4.3): z = A v_j from the
// element terms and the CGS2 passes in ONE cooperative launch, separated by
// barriers over the trajectory's blocks instead of kernel boundaries.
//
// Rows are cut into tiles of TR rows; every pass writes one partial sum per
// (column, tile) and every sum over tiles is taken in tile order, so results
// depend on the rows and TR only (a trajectory gives the same bits in any
// launch shape, alone or in a batched launch). Per step:
//   pass 1: z of the tile's rows from the element terms (node gather), h1 = V^T z
//           (with several tiles per block the gather is a sweep of its own first)
//   pass 2: z' = z - V g1, h2 = V^T z' and ||z'||^2
//   pass 3: z'' = z' - V g2 -> the new (unnormalised) basis column
// and ||z''||^2 = ||z'||^2 - ||h2||^2 (V orthonormal; the second pass removes
// only a rounding-level remainder, so the subtraction loses nothing); where it
// would cancel (||z''||^2 below 1/16 of ||z'||^2: near breakdown), pass 3 sums
// ||z''||^2 directly after all. Three barriers per step in the common case.
// Each reduction over tiles is redundant for up to kPkRedundantTiles tiles
// (every block sums every column itself, from a copy in shared memory) and
// spread over the blocks beyond (one more barrier).
// When no block has more than one tile, a block keeps its tile of V and z in
// shared memory through the three passes; the whole-solve kernel keeps it from
// one step to the next (only the new column is ever staged).
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

__device__ __forceinline__ void red_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Barrier over the nb blocks that work on one trajectory (all of a
// cooperative launch, or one trajectory's share of a batched launch; every
// block is co-resident); one object per block and launch, in registers.
// The first barrier of a launch is a generation barrier: the last block to
// arrive (atom.acq_rel) resets the arrival count and the monotone count
// `mono`, then releases the next generation, which the others acquire. Every
// later barrier k = 1, 2, ... adds one arrival to `mono` with a release
// reduction (the arriving block does not wait for a reply) and waits until
// it reads k * nb with acquire loads: one L2 round trip less than the
// generation barrier. A block's writes are ordered before its arrival by
// __syncthreads and the release; __syncthreads after the wait hands the
// acquired view to the whole block. Bounded: a block that waits `limit` polls
// records KERR_TIMEOUT in *err and goes on, so the kernel always ends; the
// host reports ETP_ERR_TIMEOUT, resets the counts and does not commit the step.
struct GridBar {
  unsigned int* count;
  unsigned int* gen;
  unsigned int* mono;
  int* err;
  int nb;
  unsigned int k;
  unsigned long long limit;

  __device__ __forceinline__ void sync() {
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long spins = 0;
      if (k == 0) {
        const unsigned int g = ld_acquire_gpu(gen);  // generation before this block arrives
        if (atom_add_acq_rel_gpu(count, 1u) == (unsigned int)nb - 1) {
          st_relaxed_gpu(count, 0u);
          st_relaxed_gpu(mono, 0u);
          st_release_gpu(gen, g + 1u);
        } else {
          while (ld_acquire_gpu(gen) == g) {
            if (++spins > limit) {
              atomicOr(err, KERR_TIMEOUT);
              break;
            }
          }
        }
      } else {
        red_release_gpu(mono, 1u);
        const unsigned int target = k * (unsigned int)nb;
        while (ld_acquire_gpu(mono) < target) {
          if (++spins > limit) {
            atomicOr(err, KERR_TIMEOUT);
            break;
          }
        }
      }
    }
    ++k;
    __syncthreads();
  }
};

// The barrier of a group whose three counter words start at `words`
// (arrivals, generation, monotone arrivals).
__device__ __forceinline__ GridBar make_grid_bar(unsigned int* words, int* err, int nb,
                                                 unsigned long long limit = kBarrierSpinLimit) {
  GridBar b;
  b.count = words;
  b.gen = words + 1;
  b.mono = words + 2;
  b.err = err;
  b.nb = nb;
  b.k = 0;
  b.limit = limit;
  return b;
}

template <typename T>
struct PkParams {
  int64_t n_nodes, nn_pad;
  const int32_t* inc_ptr;
  const int32_t* inc_idx;
  BoxInc box;             // lexicographic Q1 box: the incidences without the lists
  const T* Ye;            // element contributions of A v_j
  const T* minvsqrt;
  const uint8_t* fixed;
  const T* xb;            // bottom half of v_j (stored column)
  const double* xscale;   // column scale of v_j
  CgsParams<T> c;         // basis, z, coefficients, partials, Hessenberg, state
  const T* pbar;          // loaded state: P_bar (SoA 3*nn_pad) and the augmented entry of v_j
  const T* xi;
  unsigned int* bar;      // three counter words of the group barrier (GridBar)
  // polls before a barrier wait gives up: kBarrierSpinLimit, or the lower
  // limit a test sets (etp_debug_spin_limit) to make the wait run out. Only
  // this kernel's barriers take it: every loop bound and index here is a
  // launch parameter, so a block that leaves a barrier early computes wrong
  // values but stays in bounds and ends.
  unsigned long long spin_limit;
  // dynamic shared memory: the tile area from offset 0, then (at red_off,
  // red_bytes long) room for a copy of one pass's partial sums
  uint32_t red_off, red_bytes;
  // columns 0..res_cols-1 of this block's tile already in the tile area (the
  // whole-solve kernel, one tile per block and the same TR as the last step)
  int res_cols;
};

// Tiles of a vector of L rows, and the stride of one column of partial sums
// (even, so that every column starts on a 16-byte boundary).
__host__ __device__ constexpr int64_t pk_ntiles(int64_t L, int TR) { return L / TR; }
__host__ __device__ constexpr int64_t pk_pstride(int64_t L, int TR) { return (L / TR + 1) / 2 * 2; }

// Doubles of partial sums one persistent step of j columns needs: pass 1 (j
// columns), pass 2 (j + 1) and the direct norm of pass 3 (1).
__host__ __device__ constexpr int64_t pk_partials_count(int64_t L, int j, int TR) {
  return (2 * (int64_t)j + 2) * pk_pstride(L, TR);
}

// Bytes of the tile area: two pipeline stages of j columns and z (a single
// tile of j + 1 columns fits in it too).
template <typename T>
__host__ __device__ constexpr size_t pk_tile_bytes(int j, int TR) {
  return (2 * ((size_t)j * (TR + 1) + TR) * sizeof(T) + 15) / 16 * 16;
}

// Reductions over at most this many tiles are redundant (no barrier after them).
constexpr int64_t kPkRedundantTiles = 256;

// Tile rows for j columns of a vector of L rows: 256 where 128-row tiles would
// exceed the redundant reductions and 256-row ones do not, else the largest of
// 128, 64, 32; always with the two stages within 200 KB of shared memory
// (256-row tiles everywhere made the served batch ~10% slower: more shared
// memory per block, for no gain where the tiles outnumber the blocks anyway).
constexpr size_t kPkSmemMax = 200 * 1024;
template <typename T>
constexpr int pk_tile_rows(int j, int64_t L) {
  return (pk_ntiles(L, 128) > kPkRedundantTiles && pk_ntiles(L, 256) <= kPkRedundantTiles &&
          pk_tile_bytes<T>(j, 256) <= kPkSmemMax)
             ? 256
         : pk_tile_bytes<T>(j, 128) <= kPkSmemMax                                            ? 128
         : pk_tile_bytes<T>(j, 64) <= kPkSmemMax                                             ? 64
                                                                                             : 32;
}

// Bytes of the copy of one reduction's partials (the widest pass: j + 1 columns).
__host__ __device__ constexpr size_t pk_red_bytes(int64_t L, int j, int TR) {
  return (size_t)(j + 1) * pk_pstride(L, TR) * sizeof(double);
}

// ---- per-tile arithmetic (the same in every staging mode) ------------------

// z at one row: the top half is the bottom half of v_j times its scale; the
// bottom half is -M^-1/2 times the sum of the element terms of the node
// (incidence order) plus the load column, zero on fixed DOFs and padding nodes.
template <typename T>
__device__ __forceinline__ T gather_row(const PkParams<T>& p, int64_t row, T xs, T lx) {
  const int64_t nn = p.nn_pad, half = 3 * nn;
  if (row < half) return p.xb[row] * xs;
  const int rr = (int)(row - half), nn32 = (int)nn;  // 32-bit: short vectors only
  const int c = rr / nn32;
  const int64_t n = rr - c * nn32;
  if (n >= p.n_nodes) return T(0);
  const T a = node_sum1<T>(p.inc_ptr, p.inc_idx, p.box, p.Ye, n, c);
  const T l = p.pbar ? lx * p.pbar[c * nn + n] : T(0);
  const T s = -p.minvsqrt[n];
  return ((p.fixed[n] >> c) & 1) ? T(0) : s * a + l;
}

// z of the tile's rows r0 .. r0+TR-1 into zt (shared).
template <typename T, int TR>
__device__ __forceinline__ void tile_gather(const PkParams<T>& p, int64_t r0, T* zt, T xs, T lx) {
  for (int r = threadIdx.x; r < TR; r += blockDim.x) zt[r] = gather_row(p, r0 + r, xs, lx);
}

// zt -= V g over the tile's rows (thread r owns row r); optionally the new rows
// are written to dst (global).
template <typename T, int TR>
__device__ __forceinline__ void tile_update(const T* Vt, T* zt, int j, const T* s_g, T* dst) {
  constexpr int LD = TR + 1;
  for (int r = threadIdx.x; r < TR; r += blockDim.x) {
    T upd = T(0);
    for (int i = 0; i < j; ++i) upd += Vt[i * LD + r] * s_g[i];
    const T zn = zt[r] - upd;
    zt[r] = zn;
    if (dst) dst[r] = zn;
  }
}

// Double-length accumulator of the persistent step's sums: float-float for
// FP32 tiles (FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU, and
// these sums sit on the step's critical path), plain double for FP64 tiles.
// One value fills one 8-byte slot: (hi, lo) floats, or the double.
template <typename T>
struct Acc;

template <>
struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) { acc_add(hi, lo, x); }
  __device__ __forceinline__ void add(const Acc& o) { acc_add_pair(hi, lo, o.hi, o.lo); }
  // x^2 exactly as p + e (FMA), then added
  __device__ __forceinline__ void add_sq(float x) {
    const float p = x * x;
    const float e = fmaf(x, x, -p);
    acc_add(hi, lo, p);
    lo += e;
  }
  __device__ __forceinline__ Acc neg() const { return Acc{-hi, -lo}; }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ float tile_value() const { return hi + lo; }
  __device__ __forceinline__ void put(double* slot) const { store_partial(slot, hi, lo); }
  __device__ __forceinline__ static Acc get(const double* slot) {  // shared memory or this block's writes
    const float2 v = *reinterpret_cast<const float2*>(slot);
    return Acc{v.x, v.y};
  }
  __device__ __forceinline__ static Acc get_cg(const double* slot) {  // other blocks' writes (L2)
    const float2 v = __ldcg(reinterpret_cast<const float2*>(slot));
    return Acc{v.x, v.y};
  }
  // a * b (two-product of the leading parts plus the cross terms), normalised
  __device__ __forceinline__ static Acc mul(const Acc& a, const Acc& b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    const float s = p + e;
    return Acc{s, e - (s - p)};
  }
};

template <>
struct Acc<double> {
  double hi = 0.0;
  __device__ __forceinline__ void add(double x) { hi += x; }
  __device__ __forceinline__ void add(const Acc& o) { hi += o.hi; }
  __device__ __forceinline__ void add_sq(double x) { hi = fma(x, x, hi); }
  __device__ __forceinline__ Acc neg() const { return Acc{-hi}; }
  __device__ __forceinline__ double value() const { return hi; }
  __device__ __forceinline__ double tile_value() const { return hi; }
  __device__ __forceinline__ void put(double* slot) const { *slot = hi; }
  __device__ __forceinline__ static Acc get(const double* slot) { return Acc{*slot}; }
  __device__ __forceinline__ static Acc get_cg(const double* slot) { return Acc{__ldcg(slot)}; }
  __device__ __forceinline__ static Acc mul(const Acc& a, const Acc& b) { return Acc{a.hi * b.hi}; }
};

// Butterfly sum over a warp; lane 0's result is the one used (float-float
// additions are not symmetric in their low parts).
template <typename T>
__device__ __forceinline__ Acc<T> warp_sum_acc(Acc<T> a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Acc<T> b;
    b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
    if constexpr (sizeof(T) == 4) b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
    a.add(b);
  }
  return a;
}

// Sum over the block (128 threads): warps in order; valid in thread 0.
template <typename T>
__device__ __forceinline__ Acc<T> block_sum_acc(Acc<T> a, double* s_red) {
  a = warp_sum_acc<T>(a);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) a.put(s_red + (threadIdx.x >> 5));
  __syncthreads();
  Acc<T> r;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r.add(Acc<T>::get(s_red + w));
  return r;
}

// ||zt||^2 of the tile (squares of the stored values, fixed order) -> *out.
template <int TR, typename T>
__device__ __forceinline__ void tile_norm(const T* zt, double* out, double* s_red) {
  Acc<T> a;
  for (int r = threadIdx.x; r < TR; r += blockDim.x) a.add_sq(zt[r]);
  a = block_sum_acc<T>(a, s_red);
  if (threadIdx.x == 0) a.put(out);
}

// Sum the per-segment accumulators of the tile's dot products into one per
// column, in segment order: afterwards acc of thread i < j holds column i.
template <typename T>
__device__ __forceinline__ void combine_segments(int j, Acc<T>& acc, double* s_tmp) {
  constexpr int BD = 128;
  if (j > BD) return;  // one column (or two) per thread already
  const int tid = threadIdx.x;
  __syncthreads();
  acc.put(s_tmp + tid);
  __syncthreads();
  if (tid < j) {
    const int S = BD / j;
    Acc<T> t;
    for (int seg = 0; seg < S; ++seg) t.add(Acc<T>::get(s_tmp + seg * j + tid));
    acc = t;
  }
  __syncthreads();
}

// Dot products of the tile's z with its j columns -> out[i * ps] (column i).
// j <= 128: thread t takes column t % j over row segment t / j (cgs_segment)
// and the segments are added in order; beyond, thread i takes columns i and
// i + 128 over all rows. FP32 tiles add 16 products in FP32 before each
// float-float addition.
template <typename T, int TR>
__device__ __forceinline__ void tile_dots(const T* Vt, const T* zt, int j, double* out, int64_t ps, double* s_tmp) {
  constexpr int BD = 128, LD = TR + 1, CH = 16;
  const int tid = threadIdx.x;
  auto column = [&](const T* vr, int r_lo, int r_hi) {
    Acc<T> a;
    if (sizeof(T) == 8) {
      for (int r = r_lo; r < r_hi; ++r) a.add(vr[r] * zt[r]);
    } else {
      for (int r = r_lo; r < r_hi; r += CH) {
        T part = T(0);
#pragma unroll
        for (int u = 0; u < CH; ++u) part += vr[r + u] * zt[r + u];
        a.add(part);
      }
    }
    return a;
  };
  Acc<T> acc0, acc1;
  if (j <= BD) {
    int col, r_lo, r_hi;
    if (cgs_segment<TR>(j, tid, col, r_lo, r_hi)) acc0 = column(Vt + col * LD, r_lo, r_hi);
    combine_segments<T>(j, acc0, s_tmp);
  } else {
    if (tid < j) acc0 = column(Vt + tid * LD, 0, TR);
    if (tid + BD < j) acc1 = column(Vt + (tid + BD) * LD, 0, TR);
  }
  if (tid < j) acc0.put(out + (int64_t)tid * ps);
  if (tid + BD < j) acc1.put(out + (int64_t)(tid + BD) * ps);
}

// ---- passes ------------------------------------------------------------------

// One pass over this block's tiles. PASS 1: gather z, dot products with the j
// columns. PASS 2: update z, dot products and ||z'||^2 (column j of out).
// PASS 3: update z into the new column; with `norm`, ||z''||^2 (out[t]).
// Partial sums of tile t go to out[i * ps + t].
// One tile per block (ntiles <= nb): the tile stays in the tile area through
// the passes; pass 1 gathers z into it and stages only columns res_cols..j-1.
// Otherwise the tiles bid, bid + nb, ... go through a two-stage cp.async
// pipeline, with z (gathered beforehand by pk_gather), z' and z'' kept in the
// work vector between passes.
template <typename T, int TR, int PASS>
__device__ __forceinline__ void pk_pass(const PkParams<T>& p, unsigned char* smem_raw, const T* s_g, int bid, int nb,
                                        double* out, int64_t ps, bool norm, T xs, T lx, double* s_tmp,
                                        double* s_red) {
  constexpr int LD = TR + 1;
  const int j = p.c.j, tid = threadIdx.x;
  const int64_t L = p.c.L, ntiles = pk_ntiles(L, TR);
  T* const buf0 = reinterpret_cast<T*>(smem_raw);
  if (ntiles <= nb) {
    if (bid >= ntiles) return;
    const int64_t t = bid, r0 = t * TR;
    T* const zt = buf0 + (size_t)j * LD;
    if (PASS == 1) {
      for (int i = p.res_cols; i < j; ++i)
        for (int r = tid; r < TR; r += blockDim.x) cp_async_elem(buf0 + i * LD + r, p.c.V + (int64_t)i * L + r0 + r);
      cp_async_commit();
      tile_gather<T, TR>(p, r0, zt, xs, lx);
      cp_async_wait<0>();
      __syncthreads();
      tile_dots<T, TR>(buf0, zt, j, out + t, ps, s_tmp);
    } else {
      tile_update<T, TR>(buf0, zt, j, s_g, PASS == 3 ? p.c.vout + r0 : (T*)nullptr);
      __syncthreads();
      if (PASS == 2) {
        tile_dots<T, TR>(buf0, zt, j, out + t, ps, s_tmp);
        tile_norm<TR>(zt, out + (int64_t)j * ps + t, s_red);
      } else if (norm) {
        tile_norm<TR>(zt, out + t, s_red);
      }
    }
    return;
  }
  T* const buf1 = buf0 + (size_t)j * LD + TR;
  auto issue = [&](int64_t t, T* b) {
    const int64_t r0 = t * TR;
    for (int i = 0; i < j; ++i)
      for (int r = tid; r < TR; r += blockDim.x) cp_async_elem(b + i * LD + r, p.c.V + (int64_t)i * L + r0 + r);
    for (int r = tid; r < TR; r += blockDim.x) cp_async_elem(b + (size_t)j * LD + r, p.c.z + r0 + r);
  };
  int64_t t = bid;
  if (t < ntiles) issue(t, buf0);
  cp_async_commit();
  int stage = 0;
  for (; t < ntiles; t += nb) {
    const int64_t tn = t + nb, r0 = t * TR;
    T* const cur = stage ? buf1 : buf0;
    T* const zt = cur + (size_t)j * LD;
    if (tn < ntiles) issue(tn, stage ? buf0 : buf1);
    cp_async_commit();
    cp_async_wait<1>();  // the group of tile t has landed
    __syncthreads();
    if (PASS == 1) {
      tile_dots<T, TR>(cur, zt, j, out + t, ps, s_tmp);
    } else {
      tile_update<T, TR>(cur, zt, j, s_g, PASS == 3 ? p.c.vout + r0 : p.c.z + r0);
      __syncthreads();
      if (PASS == 2) {
        tile_dots<T, TR>(cur, zt, j, out + t, ps, s_tmp);
        tile_norm<TR>(zt, out + (int64_t)j * ps + t, s_red);
      } else if (norm) {
        tile_norm<TR>(zt, out + t, s_red);
      }
    }
    __syncthreads();  // this stage is refilled at the next iteration
    stage ^= 1;
  }
  cp_async_wait<0>();
}

// z = A v_j into the work vector over all rows (grid-stride over the group's
// blocks, independent loads in flight): the gather of the multi-tile mode,
// whose tiles would otherwise wait for one gather after another.
template <typename T>
__device__ __forceinline__ void pk_gather(const PkParams<T>& p, int bid, int nb, T xs, T lx) {
  for (int64_t row = (int64_t)bid * blockDim.x + threadIdx.x; row < p.c.L; row += (int64_t)nb * blockDim.x)
    p.c.z[row] = gather_row(p, row, xs, lx);
}

// ---- reductions over tiles -----------------------------------------------------

// Redundant: every block sums columns 0..ncol-1 of `part` ([ncol][ps], ntiles
// used) in the same order: warp w takes columns w, w+4, ...; lane k adds tiles
// k, k+32, ... in order, then the butterfly; lane 0 writes the sum to out[i].
// The partials are first copied into shared memory at `stage` when given (one
// round trip instead of one per load).
template <typename T>
__device__ __forceinline__ void pk_sum_redundant(const double* part, int64_t ntiles, int64_t ps, int ncol,
                                                 double* stage, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (stage) {
    const int64_t nchunk = (int64_t)ncol * ps / 2;  // 16-byte chunks (ps is even)
    for (int64_t c = threadIdx.x; c < nchunk; c += blockDim.x) cp_async16_cg(stage + 2 * c, part + 2 * c);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
  }
  if (stage) {
    for (int i = warp; i < ncol; i += nw) {
      Acc<T> d;
      for (int64_t t = lane; t < ntiles; t += 32) d.add(Acc<T>::get(stage + (int64_t)i * ps + t));
      d = warp_sum_acc<T>(d);
      if (lane == 0) d.put(out + i);
    }
  } else {
    // from L2: every load of CB columns in flight at once (at most kPkRedundantTiles / 32
    // per lane and column), then the same additions in the same order
    constexpr int NT = (int)(kPkRedundantTiles / 32), CB = 4;
    for (int i0 = warp * CB; i0 < ncol; i0 += nw * CB) {
      Acc<T> v[CB][NT];
#pragma unroll
      for (int c = 0; c < CB; ++c)
#pragma unroll
        for (int k = 0; k < NT; ++k) {
          const int64_t t = lane + 32 * k;
          if (i0 + c < ncol && t < ntiles) v[c][k] = Acc<T>::get_cg(part + (int64_t)(i0 + c) * ps + t);
        }
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        Acc<T> d;
#pragma unroll
        for (int k = 0; k < NT; ++k)
          if (lane + 32 * k < ntiles) d.add(v[c][k]);
        d = warp_sum_acc<T>(d);
        if (lane == 0 && i0 + c < ncol) d.put(out + i0 + c);
      }
    }
  }
  __syncthreads();
}

// Spread over the blocks: block b sums columns b, b+nb, ... (thread k adds
// tiles k, k+128, ... in order, then the block sum) and stores them in `dst`;
// after a barrier every block reads all ncol sums into `out`.
template <typename T>
__device__ __forceinline__ void pk_sum_distributed(const double* part, int64_t ntiles, int64_t ps, int ncol, int bid,
                                                   int nb, double* dst, double* out, double* s_red, GridBar& gb) {
  for (int i = bid; i < ncol; i += nb) {
    Acc<T> d;
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) d.add(Acc<T>::get_cg(part + (int64_t)i * ps + t));
    d = block_sum_acc<T>(d, s_red);
    if (threadIdx.x == 0) d.put(dst + i);
  }
  gb.sync();
  for (int i = threadIdx.x; i < ncol; i += blockDim.x) Acc<T>::get_cg(dst + i).put(out + i);
  __syncthreads();
}

// Block scratch of the persistent step, one copy per kernel whatever the tile
// rows (a function-scope shared variable of a non-template function).
struct PkScratch {
  double d[kMaxCap + 1];  // raw sums of the current pass
  double h1[kMaxCap];     // h1 (for the Hessenberg column)
  double sc[kMaxCap];     // column scales
  double red[32];
  double tmp[128];
  int pyth, flag;
};
__device__ __forceinline__ PkScratch& pk_scratch() {
  __shared__ PkScratch s;
  return s;
}
// Update coefficients in the tile precision.
template <typename T>
__device__ __forceinline__ T* pk_scratch_g() {
  __shared__ T s[kMaxCap];
  return s;
}

// Sums of the partials of one pass: redundant (from a shared-memory copy when
// the reserved area holds it) or spread over the blocks.
template <typename T>
__device__ __forceinline__ void pk_sum(const PkParams<T>& p, unsigned char* smem_raw, const double* part,
                                       int64_t ntiles, int64_t ps, int ncol, int bid, int nb, double* dst,
                                       double* out, double* s_red, GridBar& gb) {
  if (ntiles <= kPkRedundantTiles) {
    const bool fits = (size_t)ncol * ps * sizeof(double) <= p.red_bytes;
    pk_sum_redundant<T>(part, ntiles, ps, ncol, fits ? reinterpret_cast<double*>(smem_raw + p.red_off) : nullptr, out);
  } else {
    pk_sum_distributed<T>(part, ntiles, ps, ncol, bid, nb, dst, out, s_red, gb);
  }
}

// Last of n blocks to arrive at `counter` (which it resets): its writes and
// those of the n-1 blocks before it are visible to it afterwards.
__device__ __forceinline__ bool pk_elect_last(unsigned int* counter, unsigned int n, int* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int v = atomicAdd(counter, 1u);
    *s_flag = (v == n - 1);
    if (v == n - 1) atomicExch(counter, 0u);
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// One Arnoldi step of one trajectory on blocks bid = 0..nb-1 of its group.
// On return the new column is written by every block for its tiles, and one
// block (the first block without a tile, else block 0, or in the rare
// direct-norm case the last block to finish pass 3) has written column j-1 of
// H, the scale of the new column and the stop state. The caller's barrier (or
// the end of the launch) publishes them. With one tile per block, the other
// blocks without a tile only join the barriers.
template <typename T, int TR>
__device__ __forceinline__ void pk_step(const PkParams<T>& p, int bid, int nb, unsigned char* smem_raw, GridBar& gb) {
  KState* ks = p.c.ks;
  if (__ldcg(&ks->stop)) return;  // written before a barrier (or between launches): the same for every block
  using A = Acc<T>;
  constexpr int BD = 128;
  PkScratch& sc = pk_scratch();
  T* const s_g = pk_scratch_g<T>();
  double* const s_d = sc.d;    // sums of the current pass (A slots)
  double* const s_h1 = sc.h1;  // h1 (A slots)
  double* const s_sc = sc.sc;  // column scales (A slots)
  double* const s_red = sc.red;
  double* const s_tmp = sc.tmp;
  const int tid = threadIdx.x, j = p.c.j;
  const int64_t ntiles = pk_ntiles(p.c.L, TR), ps = pk_pstride(p.c.L, TR);
  const bool redundant = ntiles <= kPkRedundantTiles;
  const bool has_tile = bid < ntiles;
  // the block that writes the Hessenberg column: the first block without a tile
  // where there is one (it does the column while the others run pass 3), else block 0
  const int fin = ntiles < nb ? (int)ntiles : 0;
  const bool sums = !redundant || has_tile || bid == fin;
  double* coef = p.c.coef;
  double* part1 = p.c.partials;
  double* part2 = part1 + (int64_t)j * ps;
  double* part3 = part2 + (int64_t)(j + 1) * ps;
  // column scales, copied while pass 1 runs (FP32 tiles: the float-float pairs)
  {
    const double* src = coef + (sizeof(T) == 4 ? COEF_SCALE2 : COEF_SCALE) * COEF_STRIDE;
    for (int i = tid; i < j; i += BD) cp_async_elem(s_sc + i, src + i);
    cp_async_commit();
  }
  const T xs = (T)(*p.xscale);
  const T lx = p.pbar ? (*p.xi) * xs : T(0);
  // h = s_i d_i and g = s_i h (the update coefficient, in the tile precision)
  auto coefficients = [&](double* h_out) {
    for (int i = tid; i < j; i += BD) {
      const A si = A::get(s_sc + i);
      const A h = A::mul(si, A::get(s_d + i));
      if (h_out) h.put(h_out + i);
      s_g[i] = (T)A::mul(si, h).tile_value();
    }
  };

  // ---- pass 1: z = A v_j over the tiles, h1 = V^T z
  if (ntiles > nb) {  // several tiles per block: the gather first, in one sweep
    pk_gather<T>(p, bid, nb, xs, lx);
    gb.sync();
  }
  pk_pass<T, TR, 1>(p, smem_raw, s_g, bid, nb, part1, ps, false, xs, lx, s_tmp, s_red);
  gb.sync();
  if (sums) {
    pk_sum<T>(p, smem_raw, part1, ntiles, ps, j, bid, nb, coef + COEF_H1 * COEF_STRIDE, s_d, s_red, gb);
    cp_async_wait<0>();  // the scales
    __syncthreads();
    coefficients(s_h1);
    __syncthreads();
  } else {
    cp_async_wait<0>();  // no copy left in flight in a block without a tile
  }

  // ---- pass 2: z' = z - V g1, h2 = V^T z', ||z'||^2
  pk_pass<T, TR, 2>(p, smem_raw, s_g, bid, nb, part2, ps, false, xs, lx, s_tmp, s_red);
  gb.sync();
  if (!sums) return;
  pk_sum<T>(p, smem_raw, part2, ntiles, ps, j + 1, bid, nb, coef + COEF_H2 * COEF_STRIDE, s_d, s_red, gb);
  // ||z''||^2 = ||z'||^2 - sum h2_i^2 (warp 0, fixed order); kept unless it cancels
  if (tid < 32) {
    A q;
    for (int i = tid; i < j; i += 32) {
      const A h = A::mul(A::get(s_sc + i), A::get(s_d + i));
      q.add(A::mul(h, h));
    }
    q = warp_sum_acc<T>(q);
    if (tid == 0) {
      A n2 = A::get(s_d + j);
      const double n1 = n2.value();
      n2.add(q.neg());
      const double v = n2.value();
      sc.pyth = (v > 0.0625 * n1) ? 1 : 0;  // false for a non-finite value
      s_tmp[0] = v;
    }
  }
  coefficients(nullptr);
  __syncthreads();
  const bool pyth = sc.pyth != 0;
  double n2 = s_tmp[0];
  __syncthreads();

  // ---- pass 3: z'' = z' - V g2 -> new basis column (and its norm if needed)
  pk_pass<T, TR, 3>(p, smem_raw, s_g, bid, nb, part3, ps, !pyth, xs, lx, s_tmp, s_red);
  if (!pyth) {
    // direct norm: the last of the blocks with tiles sums the tiles' norms
    if (!has_tile) return;
    if (!pk_elect_last(p.c.counter + 4, (unsigned int)(ntiles < nb ? ntiles : nb), &sc.flag)) return;
    A a;
    for (int64_t t = tid; t < ntiles; t += BD) a.add(A::get_cg(part3 + t));
    a = block_sum_acc<T>(a, s_red);
    if (tid == 0) s_tmp[0] = a.value();
    __syncthreads();
    n2 = s_tmp[0];
  } else if (bid != fin) {
    return;
  }
  // ---- Hessenberg column, breakdown test, scale of the new column
  const int col = j - 1;
  A hsq;
  for (int i = tid; i < j; i += BD) {
    A h = A::get(s_h1 + i);
    h.add(A::mul(A::get(s_sc + i), A::get(s_d + i)));
    p.c.H[i + (int64_t)col * p.c.ldH] = h.value();
    hsq.add(A::mul(h, h));
  }
  const double colsum = block_sum_acc<T>(hsq, s_red).value();
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
      const double s = 1.0 / hn;
      coef[COEF_SCALE * COEF_STRIDE + j] = s;
      store_scale_pair(coef + COEF_SCALE2 * COEF_STRIDE + j, s);
    }
    ks->hnorm2 = hn2 + hn * hn;
    if (ks->err & KERR_TIMEOUT) ks->stop = 1;
  }
}

// Dynamic shared memory of one persistent step of j columns over vectors of L
// rows with TR-row tiles: the tile area, then (where the reduction is redundant
// and it fits) room for the copy of one pass's partial sums. Sets q's offsets.
template <typename T>
inline size_t pk_step_smem(int64_t L, int j, int TR, PkParams<T>& q) {
  const size_t tile = pk_tile_bytes<T>(j, TR);
  size_t red = 0;
  if (pk_ntiles(L, TR) <= kPkRedundantTiles && tile + pk_red_bytes(L, j, TR) <= kPkSmemMax) red = pk_red_bytes(L, j, TR);
  q.red_off = (uint32_t)tile;
  q.red_bytes = (uint32_t)red;
  q.res_cols = 0;
  return tile + red > 1024 ? tile + red : 1024;
}

// Co-resident blocks per SM (at most 2) of a persistent-step kernel with this
// much dynamic shared memory (solve.cu; cached per kernel and size).
int pk_blocks_per_sm(const void* fn, size_t smem);
// Lets a persistent-step kernel use all dynamic shared memory beside its static (solve.cu).
void pk_allow_smem(const void* fn);
// Dynamic shared memory per block that still fits two blocks per SM (solve.cu).
size_t pk_two_per_sm_smem(const void* fn);

template <typename T, int TR>
static __global__ void __launch_bounds__(128) k_arnoldi_step_pk(PkParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GridBar gb = make_grid_bar(p.bar, &p.c.ks->err, (int)gridDim.x, p.spin_limit);
  pk_step<T, TR>(p, blockIdx.x, gridDim.x, smem_raw, gb);
}

// Ragged batch: the Arnoldi steps of up to kMaxBatch trajectories (each its
// own mesh, size and column count j; one tile size per launch) in one
// cooperative launch. Trajectory i owns blocks off[i] .. off[i+1]-1 and
// synchronises only them.
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
  const PkParams<T>& q = b.item[i];
  const int nb = b.off[i + 1] - b.off[i];
  GridBar gb = make_grid_bar(q.bar, &q.c.ks->err, nb, q.spin_limit);
  pk_step<T, TR>(q, (int)blockIdx.x - b.off[i], nb, smem_raw, gb);
}

}  // namespace etp
