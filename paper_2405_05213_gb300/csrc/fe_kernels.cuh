// Finite-element kernels: operator apply z = A v (Section 2.3), GLL mass
// (Section 2.2), element geometry, stored energy (Section 5.2).
#pragma once

#include "etp_internal.cuh"
#include "material.cuh"

namespace etp {

// ------------------------------------------------------------ 1D Lagrange bases
// Nodes at -1 (+0) +1; Gauss-Legendre points with P+1 points per axis.
template <int P, typename T>
__host__ __device__ __forceinline__ T gauss_pt(int i) {
  if (P == 1) return i == 0 ? T(-0.57735026918962576451) : T(0.57735026918962576451);
  return i == 0 ? T(-0.77459666924148337704) : (i == 1 ? T(0) : T(0.77459666924148337704));
}
template <int P, typename T>
__host__ __device__ __forceinline__ T gauss_w(int i) {
  if (P == 1) return T(1);
  return i == 1 ? T(8.0 / 9.0) : T(5.0 / 9.0);
}
template <int P, typename T>
__host__ __device__ __forceinline__ T lag(int a, T x) {
  if (P == 1) return a == 0 ? T(0.5) * (T(1) - x) : T(0.5) * (T(1) + x);
  if (a == 0) return T(0.5) * x * (x - T(1));
  if (a == 1) return (T(1) - x) * (T(1) + x);
  return T(0.5) * x * (x + T(1));
}
template <int P, typename T>
__host__ __device__ __forceinline__ T dlag(int a, T x) {
  if (P == 1) return a == 0 ? T(-0.5) : T(0.5);
  if (a == 0) return x - T(0.5);
  if (a == 1) return T(-2) * x;
  return x + T(0.5);
}
// GLL weights at the nodes (2-point and 3-point Lobatto)
template <int P>
__host__ __device__ __forceinline__ double gll_w(int a) {
  if (P == 1) return 1.0;
  return a == 1 ? 4.0 / 3.0 : 1.0 / 3.0;
}

template <int P>
struct ElemTraits {
  static constexpr int N1 = P + 1;
  static constexpr int NEN = N1 * N1 * N1;
  static constexpr int NQ = NEN;
  static constexpr int TEAM = (P == 1) ? 8 : 32;
  static constexpr int BLOCK = 128;
  static constexpr int EPB = BLOCK / TEAM;  // elements per block
};

template <typename T>
struct ApplyParams {
  int64_t n_elems, nn_pad;
  const int32_t* conn;
  const T* x;            // top half of the input Krylov vector (3 SoA components)
  const double* xscale;  // device pointer to the column scale of x
  const T* minvsqrt;     // 1/sqrt(m) per node
  const T* geo;          // general meshes: per (e,q) Jinv (row-major) + dV
  T hinv[3];             // box: 2/h per axis
  T dvbox;               // box: hx*hy*hz/8
  const float* escale;   // per element or null
  const T* us0;          // frozen displacements (physical, SoA)
  const T* us1;
  T c0, c1;
  T prm[kMaxParams];
  T* Ye;                 // out: (e, A, comp)
  int* err;
  const int* stop;       // skip the launch when *stop != 0 (may be null)
};

// Team-per-element apply of P_lin. Phase 1: lane = Gauss point q computes
// grad x and grad u* there, the secant stress and P dV. Phase 2: lane = node A
// sums P : grad N_A over the Gauss points.
template <int P, typename T, int KIND, bool BOX, int NS>
static __global__ void __launch_bounds__(128) k_elem_apply(ApplyParams<T> p) {
  using Tr = ElemTraits<P>;
  constexpr int N1 = Tr::N1, NEN = Tr::NEN, NQ = Tr::NQ, TEAM = Tr::TEAM, EPB = Tr::EPB;
  __shared__ T s_x[EPB][NEN * 3];
  __shared__ T s_u[EPB][NS > 0 ? NS : 1][NEN * 3];
  __shared__ T s_P[EPB][NQ * 9];
  __shared__ T s_J[EPB][BOX ? 1 : NQ * 9];
  if (p.stop && *p.stop) return;
  const int team = threadIdx.x / TEAM, lane = threadIdx.x % TEAM;
  const int64_t e = (int64_t)blockIdx.x * EPB + team;
  const bool active = e < p.n_elems;
  const T xs = (T)(*p.xscale);
  if (active) {
    for (int A = lane; A < NEN; A += TEAM) {
      const int node = p.conn[e * NEN + A];
      const T s = p.minvsqrt[node] * xs;
#pragma unroll
      for (int c = 0; c < 3; ++c) s_x[team][A * 3 + c] = p.x[c * p.nn_pad + node] * s;
      if (NS > 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) s_u[team][0][A * 3 + c] = p.us0[c * p.nn_pad + node];
      }
      if (NS > 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) s_u[team][NS - 1][A * 3 + c] = p.us1[c * p.nn_pad + node];
      }
    }
  }
  __syncthreads();
  // ---- phase 1: Gauss point q = lane
  if (active && lane < NQ) {
    const int q = lane;
    const int qx = q % N1, qy = (q / N1) % N1, qz = q / (N1 * N1);
    T Nx[N1], Ny[N1], Nz[N1], dx[N1], dy[N1], dz[N1];
    const T xq = gauss_pt<P, T>(qx), yq = gauss_pt<P, T>(qy), zq = gauss_pt<P, T>(qz);
#pragma unroll
    for (int a = 0; a < N1; ++a) {
      Nx[a] = lag<P, T>(a, xq); dx[a] = dlag<P, T>(a, xq);
      Ny[a] = lag<P, T>(a, yq); dy[a] = dlag<P, T>(a, yq);
      Nz[a] = lag<P, T>(a, zq); dz[a] = dlag<P, T>(a, zq);
    }
    T Ji[9];
    T dV;
    if (BOX) {
      dV = p.dvbox * gauss_w<P, T>(qx) * gauss_w<P, T>(qy) * gauss_w<P, T>(qz);
    } else {
      const T* g = p.geo + (e * NQ + q) * 10;
#pragma unroll
      for (int i = 0; i < 9; ++i) { Ji[i] = g[i]; s_J[team][q * 9 + i] = Ji[i]; }
      dV = g[9];
    }
    T G[9], D0[9], D1[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) { G[i] = T(0); D0[i] = T(0); D1[i] = T(0); }
#pragma unroll
    for (int c = 0; c < N1; ++c)
#pragma unroll
      for (int b = 0; b < N1; ++b)
#pragma unroll
        for (int a = 0; a < N1; ++a) {
          const int A = a + N1 * (b + N1 * c);
          const T r0 = dx[a] * Ny[b] * Nz[c], r1 = Nx[a] * dy[b] * Nz[c], r2 = Nx[a] * Ny[b] * dz[c];
          T g0, g1, g2;
          if (BOX) {
            g0 = r0 * p.hinv[0]; g1 = r1 * p.hinv[1]; g2 = r2 * p.hinv[2];
          } else {  // dN/dX_i = sum_J dN/dxi_J Jinv_{J i}
            g0 = r0 * Ji[0] + r1 * Ji[3] + r2 * Ji[6];
            g1 = r0 * Ji[1] + r1 * Ji[4] + r2 * Ji[7];
            g2 = r0 * Ji[2] + r1 * Ji[5] + r2 * Ji[8];
          }
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const T xi = s_x[team][A * 3 + i];
            G[3 * i + 0] += xi * g0; G[3 * i + 1] += xi * g1; G[3 * i + 2] += xi * g2;
            if (NS > 0) {
              const T ui = s_u[team][0][A * 3 + i];
              D0[3 * i + 0] += ui * g0; D0[3 * i + 1] += ui * g1; D0[3 * i + 2] += ui * g2;
            }
            if (NS > 1) {
              const T vi = s_u[team][NS - 1][A * 3 + i];
              D1[3 * i + 0] += vi * g0; D1[3 * i + 1] += vi * g1; D1[3 * i + 2] += vi * g2;
            }
          }
        }
    T Pq[9];
    if (KIND == MAT_LINEAR) {
      linear_stress(p.prm, G, Pq);
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) Pq[i] = T(0);
      Frozen<T> fz;
      bool ok = frozen_prepare<T, KIND>(p.prm, D0, fz);
      if (ok) plin_add<T, KIND>(fz, G, NS > 1 ? p.c0 : T(1), Pq);
      if (NS > 1) {
        ok = ok && frozen_prepare<T, KIND>(p.prm, D1, fz);
        if (ok) plin_add<T, KIND>(fz, G, p.c1, Pq);
      }
      if (!ok) {
        atomicOr(p.err, KERR_INVERTED);
#pragma unroll
        for (int i = 0; i < 9; ++i) Pq[i] = T(0);
      }
    }
    const T w = dV * (p.escale ? (T)p.escale[e] : T(1));
#pragma unroll
    for (int i = 0; i < 9; ++i) s_P[team][q * 9 + i] = Pq[i] * w;
  }
  __syncthreads();
  // ---- phase 2: node A = lane
  if (active && lane < NEN) {
    const int A = lane;
    const int a = A % N1, b = (A / N1) % N1, c = A / (N1 * N1);
    T out0 = T(0), out1 = T(0), out2 = T(0);
#pragma unroll
    for (int qz = 0; qz < N1; ++qz)
#pragma unroll
      for (int qy = 0; qy < N1; ++qy)
#pragma unroll
        for (int qx = 0; qx < N1; ++qx) {
          const int q = qx + N1 * (qy + N1 * qz);
          const T xq = gauss_pt<P, T>(qx), yq = gauss_pt<P, T>(qy), zq = gauss_pt<P, T>(qz);
          const T r0 = dlag<P, T>(a, xq) * lag<P, T>(b, yq) * lag<P, T>(c, zq);
          const T r1 = lag<P, T>(a, xq) * dlag<P, T>(b, yq) * lag<P, T>(c, zq);
          const T r2 = lag<P, T>(a, xq) * lag<P, T>(b, yq) * dlag<P, T>(c, zq);
          T g0, g1, g2;
          if (BOX) {
            g0 = r0 * p.hinv[0]; g1 = r1 * p.hinv[1]; g2 = r2 * p.hinv[2];
          } else {
            const T* Ji = &s_J[team][q * 9];
            g0 = r0 * Ji[0] + r1 * Ji[3] + r2 * Ji[6];
            g1 = r0 * Ji[1] + r1 * Ji[4] + r2 * Ji[7];
            g2 = r0 * Ji[2] + r1 * Ji[5] + r2 * Ji[8];
          }
          const T* Pq = &s_P[team][q * 9];
          out0 += Pq[0] * g0 + Pq[1] * g1 + Pq[2] * g2;
          out1 += Pq[3] * g0 + Pq[4] * g1 + Pq[5] * g2;
          out2 += Pq[6] * g0 + Pq[7] * g1 + Pq[8] * g2;
        }
    T* y = p.Ye + (e * NEN + A) * 3;
    y[0] = out0; y[1] = out1; y[2] = out2;
  }
}

// z = A v for v = [a; b]: z_top = s b, z_bot = -M^{-1/2} sum_e (element terms).
// Each node sums its incident element contributions in ascending order.
template <typename T>
static __global__ void k_gather_apply(int64_t n_nodes, int64_t nn_pad, const int32_t* __restrict__ inc_ptr,
                               const int32_t* __restrict__ inc_idx, const T* __restrict__ Ye,
                               const T* __restrict__ minvsqrt, const uint8_t* __restrict__ fixed,
                               const T* __restrict__ xb, const double* xscale, T* __restrict__ z,
                               const int* stop) {
  if (stop && *stop) return;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn_pad) return;
  T* zt = z;
  T* zb = z + 3 * nn_pad;
  if (n >= n_nodes) {
#pragma unroll
    for (int c = 0; c < 3; ++c) { zt[c * nn_pad + n] = T(0); zb[c * nn_pad + n] = T(0); }
    return;
  }
  const T xs = (T)(*xscale);
  T acc0 = T(0), acc1 = T(0), acc2 = T(0);
  for (int k = inc_ptr[n]; k < inc_ptr[n + 1]; ++k) {
    const T* y = Ye + (int64_t)inc_idx[k] * 3;
    acc0 += y[0]; acc1 += y[1]; acc2 += y[2];
  }
  const T s = -minvsqrt[n];
  const uint8_t f = fixed[n];
  zb[n] = (f & 1) ? T(0) : s * acc0;
  zb[nn_pad + n] = (f & 2) ? T(0) : s * acc1;
  zb[2 * nn_pad + n] = (f & 4) ? T(0) : s * acc2;
#pragma unroll
  for (int c = 0; c < 3; ++c) zt[c * nn_pad + n] = xb[c * nn_pad + n] * xs;
}

}  // namespace etp
