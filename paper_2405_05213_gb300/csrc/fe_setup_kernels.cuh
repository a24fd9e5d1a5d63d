// Mesh set-up kernels: element geometry at the Gauss points, the GLL diagonal
// mass (Section 2.2, closing paragraph) and the stored energy (Section 5.2).
#pragma once

#include "fe_kernels.cuh"
#include "krylov_kernels.cuh"

namespace etp {

// Jacobian J_{iJ} = dX_i/dxi_J at reference point (x, y, z) from the element's node coordinates.
template <int P>
__device__ __forceinline__ void jacobian_at(const double* __restrict__ coords, const int32_t* __restrict__ en,
                                            double x, double y, double z, double* J) {
  constexpr int N1 = P + 1;
#pragma unroll
  for (int i = 0; i < 9; ++i) J[i] = 0.0;
  for (int c = 0; c < N1; ++c)
    for (int b = 0; b < N1; ++b)
      for (int a = 0; a < N1; ++a) {
        const int A = a + N1 * (b + N1 * c);
        const double r0 = dlag<P, double>(a, x) * lag<P, double>(b, y) * lag<P, double>(c, z);
        const double r1 = lag<P, double>(a, x) * dlag<P, double>(b, y) * lag<P, double>(c, z);
        const double r2 = lag<P, double>(a, x) * lag<P, double>(b, y) * dlag<P, double>(c, z);
        const double* X = coords + 3 * (int64_t)en[A];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          J[3 * i + 0] += X[i] * r0;
          J[3 * i + 1] += X[i] * r1;
          J[3 * i + 2] += X[i] * r2;
        }
      }
}

// Per (element, Gauss point): J^{-1} (row-major) and dV = w detJ, in FP64 and FP32.
template <int P>
static __global__ void k_geometry(int64_t n_elems, const double* __restrict__ coords, const int32_t* __restrict__ conn,
                           double* __restrict__ geo64, float* __restrict__ geo32, int* err) {
  constexpr int N1 = P + 1, NQ = N1 * N1 * N1;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_elems * NQ) return;
  const int64_t e = id / NQ;
  const int q = (int)(id % NQ);
  const int qx = q % N1, qy = (q / N1) % N1, qz = q / (N1 * N1);
  double J[9];
  jacobian_at<P>(coords, conn + e * NQ, gauss_pt<P, double>(qx), gauss_pt<P, double>(qy),
                 gauss_pt<P, double>(qz), J);
  const double det = det3(J);
  if (!(det > 0.0)) atomicOr(err, 1);
  double C[9];
  cof3(J, C);
  double* g = geo64 + id * 10;
  float* h = geo32 + id * 10;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double v = C[3 * k + i] / det;  // inverse = cof^T / det
      g[3 * i + k] = v;
      h[3 * i + k] = (float)v;
    }
  const double dV = det * gauss_w<P, double>(qx) * gauss_w<P, double>(qy) * gauss_w<P, double>(qz);
  g[9] = dV;
  h[9] = (float)dV;
}

// Mass contribution rho * w_GLL(A) * detJ(xi_A) of each (element, local node).
template <int P>
static __global__ void k_mass_contrib(int64_t n_elems, const double* __restrict__ coords, const int32_t* __restrict__ conn,
                               double rho, int box, double box_det, double* __restrict__ mc, int* err) {
  constexpr int N1 = P + 1, NEN = N1 * N1 * N1;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n_elems * NEN) return;
  const int64_t e = id / NEN;
  const int A = (int)(id % NEN);
  const int a = A % N1, b = (A / N1) % N1, c = A / (N1 * N1);
  double det = box_det;
  if (!box) {
    double J[9];
    const double xa = -1.0 + 2.0 * a / P, yb = -1.0 + 2.0 * b / P, zc = -1.0 + 2.0 * c / P;
    jacobian_at<P>(coords, conn + e * NEN, xa, yb, zc, J);
    det = det3(J);
    if (!(det > 0.0)) atomicOr(err, 1);
  }
  mc[id] = rho * gll_w<P>(a) * gll_w<P>(b) * gll_w<P>(c) * det;
}

// Per-node sum of (element, local node) scalars over the incidence lists.
static __global__ void k_gather_scalar(int64_t n_nodes, const int32_t* __restrict__ inc_ptr,
                                const int32_t* __restrict__ inc_idx, const double* __restrict__ vals,
                                double* __restrict__ out) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  double s = 0.0;
  for (int k = inc_ptr[n]; k < inc_ptr[n + 1]; ++k) s += vals[inc_idx[k]];
  out[n] = s;
}

static __global__ void k_mass_finish(int64_t n_nodes, int64_t nn_pad, const double* __restrict__ m,
                              double* __restrict__ msqrt, double* __restrict__ minv64,
                              float* __restrict__ minv32) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn_pad) return;
  double s = 0.0, si = 0.0;
  if (n < n_nodes) {
    s = sqrt(m[n]);
    si = 1.0 / s;
  }
  msqrt[n] = s;
  minv64[n] = si;
  minv32[n] = (float)si;
}

// Stored energy sum_e sum_q psi(F) w detJ (times the element scale), FP64,
// from w_bar's displacement part. One thread per element; block partials.
template <int P>
static __global__ void __launch_bounds__(128) k_energy_elem(int64_t n_elems, int64_t nn_pad, const int32_t* __restrict__ conn,
                                                     const double* __restrict__ w, const double* __restrict__ minvsqrt,
                                                     const double* __restrict__ geo64, int box, double hx, double hy,
                                                     double hz, const float* __restrict__ escale, int kind, Prm8 prm,
                                                     double* partials) {
  constexpr int N1 = P + 1, NEN = N1 * N1 * N1, NQ = NEN;
  __shared__ double s_red[32];
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elems;
       e += (int64_t)gridDim.x * blockDim.x) {
    double ue[NEN * 3];
    for (int A = 0; A < NEN; ++A) {
      const int n = conn[e * NEN + A];
      const double s = minvsqrt[n];
      for (int c = 0; c < 3; ++c) ue[A * 3 + c] = w[c * nn_pad + n] * s;
    }
    double pe = 0.0;
    for (int q = 0; q < NQ; ++q) {
      const int qx = q % N1, qy = (q / N1) % N1, qz = q / (N1 * N1);
      const double x = gauss_pt<P, double>(qx), y = gauss_pt<P, double>(qy), z = gauss_pt<P, double>(qz);
      double Ji[9], dV;
      if (box) {
        for (int i = 0; i < 9; ++i) Ji[i] = 0.0;
        Ji[0] = 2.0 / hx; Ji[4] = 2.0 / hy; Ji[8] = 2.0 / hz;
        dV = hx * hy * hz / 8.0 * gauss_w<P, double>(qx) * gauss_w<P, double>(qy) * gauss_w<P, double>(qz);
      } else {
        const double* g = geo64 + (e * NQ + q) * 10;
        for (int i = 0; i < 9; ++i) Ji[i] = g[i];
        dV = g[9];
      }
      double D[9];
      for (int i = 0; i < 9; ++i) D[i] = 0.0;
      for (int A = 0; A < NEN; ++A) {
        const int a = A % N1, b = (A / N1) % N1, c = A / (N1 * N1);
        const double r0 = dlag<P, double>(a, x) * lag<P, double>(b, y) * lag<P, double>(c, z);
        const double r1 = lag<P, double>(a, x) * dlag<P, double>(b, y) * lag<P, double>(c, z);
        const double r2 = lag<P, double>(a, x) * lag<P, double>(b, y) * dlag<P, double>(c, z);
        const double g0 = r0 * Ji[0] + r1 * Ji[3] + r2 * Ji[6];
        const double g1 = r0 * Ji[1] + r1 * Ji[4] + r2 * Ji[7];
        const double g2 = r0 * Ji[2] + r1 * Ji[5] + r2 * Ji[8];
        for (int i = 0; i < 3; ++i) {
          D[3 * i + 0] += ue[A * 3 + i] * g0;
          D[3 * i + 1] += ue[A * 3 + i] * g1;
          D[3 * i + 2] += ue[A * 3 + i] * g2;
        }
      }
      pe += psi_of(kind, prm.v, D) * dV;
    }
    acc += pe * (escale ? (double)escale[e] : 1.0);
  }
  const double s = block_sum(acc, s_red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

static __global__ void k_sum_partials(int n, const double* partials, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partials[i];
    *out = s;
  }
}

}  // namespace etp
