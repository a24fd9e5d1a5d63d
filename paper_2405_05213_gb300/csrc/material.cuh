// Device constitutive laws and the frozen-coefficient secant split H(u*).
//
// Section 2.1 (Eq. "Constitutive equation"): S = dpsi/dE, E = (F^T F - I)/2.
// Section 2.3 (Eq. "discrete dynamic equilibrium using H"): R(u) = H(u) u.
// Appendix A.1 (St. Venant-Kirchhoff), A.2 (Yeoh, frozen alpha_e, beta_e and
// the matrix P_e with det F - 1 = P_e : grad u); Neo-Hookean and
// Mooney-Rivlin follow the same construction.
//
// The secant first Piola stress is linear in its argument G = grad x:
//   E_lin(G) = sym(G) + sym(D*^T G)/2,     j_lin(G) = P_e(D*) : G,
//   P_lin(G) = F* S_lin(G),
// with every nonlinear coefficient of S frozen at u*, so that
// P_lin(D*) = P(F*) and H(u*) u* = R(u*).
#pragma once

#include <math.h>

namespace etp {

enum : int { MAT_LINEAR = 0, MAT_NEOHOOKE = 1, MAT_MOONEY_RIVLIN = 2, MAT_SVK = 3, MAT_YEOH = 4 };
// Internal operator kind (not a material of etp_material_set): the consistent
// tangent dP/dF of Saint Venant-Kirchhoff at the stored state, for the Newton
// iterations of the nonlinear Newmark-beta step; same stored fields as MAT_SVK.
constexpr int MAT_SVK_TANGENT = 5;
__host__ __device__ constexpr bool svk_fields(int kind) { return kind == MAT_SVK || kind == MAT_SVK_TANGENT; }

template <typename T>
__host__ __device__ __forceinline__ T tr3(const T* A) { return A[0] + A[4] + A[8]; }

template <typename T>
__host__ __device__ __forceinline__ T det3(const T* A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// cof(A)_ij = (-1)^(i+j) minor_ij, row-major
template <typename T>
__host__ __device__ __forceinline__ void cof3(const T* A, T* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      C[3 * i + j] = A[3 * i1 + j1] * A[3 * i2 + j2] - A[3 * i1 + j2] * A[3 * i2 + j1];
    }
  }
}

template <typename T>
__host__ __device__ __forceinline__ void matmul3(const T* A, const T* B, T* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// log(J)/(J-1), continuous at J = 1
template <typename T>
__device__ __forceinline__ T log_ratio(T J) {
  const T x = J - T(1);
  const T small = sizeof(T) == 8 ? T(1e-8) : T(1e-4);
  if (fabs(x) < small) return T(1) - x / T(2) + x * x / T(3);
  return log1p(x) / x;
}

// J^(-2/3)
template <typename T>
__device__ __forceinline__ T jm23(T J) {
  const T c = cbrt(J);
  return T(1) / (c * c);
}

// Coefficients of the secant stress frozen at F* = I + D*.
template <typename T>
struct Frozen {
  T F[9];   // F*
  T Ds[9];  // D* = grad u*
  T Ci[9];  // C*^{-1}
  T Pe[9];  // P_e(D*)
  T Es[9];  // E* (Mooney-Rivlin)
  T k1, k2, k3;
};

// Returns false if det F* <= 0 (inverted element).
template <typename T, int KIND>
__device__ __forceinline__ bool frozen_prepare(const T* __restrict__ prm, const T* Ds, Frozen<T>& z) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    z.Ds[i] = Ds[i];
    z.F[i] = Ds[i] + ((i % 4 == 0) ? T(1) : T(0));
  }
  T C[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = z.F[i] * z.F[j] + z.F[3 + i] * z.F[3 + j] + z.F[6 + i] * z.F[6 + j];
  const T J = det3(z.F);
  if (!(J > T(0))) return false;
  T cC[9];
  cof3(C, cC);  // C symmetric: C^{-1} = cof(C) / det C
  const T idet = T(1) / (J * J);
#pragma unroll
  for (int i = 0; i < 9; ++i) z.Ci[i] = cC[i] * idet;
  T cD[9];
  cof3(Ds, cD);
  const T trD = tr3(Ds);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      z.Pe[3 * i + j] = (i == j ? T(1) + T(0.5) * trD : T(0)) - T(0.5) * Ds[3 * j + i] +
                        cD[3 * i + j] / T(3);
  if (KIND == MAT_NEOHOOKE) {
    z.k1 = T(2) * prm[0];               // 2 mu
    z.k2 = prm[1] * log_ratio(J);       // lambda ln J / (J - 1)
  } else if (KIND == MAT_MOONEY_RIVLIN) {
    const T a = jm23(J);
    z.k1 = T(2) * prm[0] * a;           // 2 C10 J^{-2/3}
    z.k2 = T(2) * prm[1] * a * a;       // 2 C01 J^{-4/3}
    z.k3 = prm[2] * J;                  // kappa J
#pragma unroll
    for (int i = 0; i < 9; ++i) z.Es[i] = T(0.5) * (C[i] - ((i % 4 == 0) ? T(1) : T(0)));
  } else if (svk_fields(KIND)) {
    z.k1 = prm[0];  // lambda
    z.k2 = prm[1];  // mu
  } else if (KIND == MAT_YEOH) {
    const T a = jm23(J);
    const T x = a * tr3(C) - T(3);
    z.k1 = T(2) * a * (prm[0] + T(2) * prm[1] * x + T(3) * prm[2] * x * x);  // alpha_e
    z.k2 = T(2) / prm[3] * J;                                                // beta_e
  }
  return true;
}

// Frozen coefficients stored per Gauss point for a whole Krylov solve: the
// state u* is fixed while the Arnoldi process runs, so F*, C*^-1, P_e(D*) and
// the scalar factors are evaluated once (k_frozen_build) and every apply only
// loads them. Fields, each a separate plane of one value per (element, point):
//   D* (9); unless SVK: C*^-1 (6, symmetric: 00 01 02 11 12 22), P_e (9);
//   Neo-Hooke: k2; Mooney-Rivlin: E* (6, symmetric), k1, k2, k3; Yeoh: k1, k2.
// Constant factors (2 mu for Neo-Hooke, lambda and mu for SVK) come from prm.
template <int KIND>
__host__ __device__ constexpr int frozen_nf() {
  return KIND == MAT_LINEAR ? 0
         : svk_fields(KIND) ? 9
         : KIND == MAT_NEOHOOKE ? 25
         : KIND == MAT_MOONEY_RIVLIN ? 33
                                     : 26;  // Yeoh
}
inline int frozen_nf_of(int kind) {
  switch (kind) {
    case MAT_LINEAR: return frozen_nf<MAT_LINEAR>();
    case MAT_SVK: return frozen_nf<MAT_SVK>();
    case MAT_SVK_TANGENT: return frozen_nf<MAT_SVK_TANGENT>();
    case MAT_NEOHOOKE: return frozen_nf<MAT_NEOHOOKE>();
    case MAT_MOONEY_RIVLIN: return frozen_nf<MAT_MOONEY_RIVLIN>();
    default: return frozen_nf<MAT_YEOH>();
  }
}

// Write the fields of z (or zeros when `ok` is false) at base[f * stride].
template <typename T, int KIND>
__device__ __forceinline__ void frozen_store(const Frozen<T>& z, bool ok, T* base, int64_t stride) {
  constexpr int NF = frozen_nf<KIND>();
  T v[NF > 0 ? NF : 1];
  int f = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) v[f++] = z.Ds[i];
  if (!svk_fields(KIND)) {
    v[f++] = z.Ci[0]; v[f++] = z.Ci[1]; v[f++] = z.Ci[2]; v[f++] = z.Ci[4]; v[f++] = z.Ci[5]; v[f++] = z.Ci[8];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[f++] = z.Pe[i];
  }
  if (KIND == MAT_NEOHOOKE) v[f++] = z.k2;
  if (KIND == MAT_MOONEY_RIVLIN) {
    v[f++] = z.Es[0]; v[f++] = z.Es[1]; v[f++] = z.Es[2]; v[f++] = z.Es[4]; v[f++] = z.Es[5]; v[f++] = z.Es[8];
    v[f++] = z.k1; v[f++] = z.k2; v[f++] = z.k3;
  }
  if (KIND == MAT_YEOH) { v[f++] = z.k1; v[f++] = z.k2; }
#pragma unroll
  for (int i = 0; i < NF; ++i) base[(int64_t)i * stride] = ok ? v[i] : T(0);
}

// Inverse of frozen_store (fills every field plin_add reads).
template <typename T, int KIND>
__device__ __forceinline__ void frozen_load(const T* __restrict__ base, int64_t stride, const T* __restrict__ prm,
                                            Frozen<T>& z) {
  int f = 0;
  auto ld = [&]() { return base[(int64_t)(f++) * stride]; };
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    z.Ds[i] = ld();
    z.F[i] = z.Ds[i] + ((i % 4 == 0) ? T(1) : T(0));
  }
  if (!svk_fields(KIND)) {
    const T c00 = ld(), c01 = ld(), c02 = ld(), c11 = ld(), c12 = ld(), c22 = ld();
    z.Ci[0] = c00; z.Ci[1] = c01; z.Ci[2] = c02;
    z.Ci[3] = c01; z.Ci[4] = c11; z.Ci[5] = c12;
    z.Ci[6] = c02; z.Ci[7] = c12; z.Ci[8] = c22;
#pragma unroll
    for (int i = 0; i < 9; ++i) z.Pe[i] = ld();
  }
  if (KIND == MAT_NEOHOOKE) {
    z.k1 = T(2) * prm[0];
    z.k2 = ld();
  } else if (KIND == MAT_MOONEY_RIVLIN) {
    const T e00 = ld(), e01 = ld(), e02 = ld(), e11 = ld(), e12 = ld(), e22 = ld();
    z.Es[0] = e00; z.Es[1] = e01; z.Es[2] = e02;
    z.Es[3] = e01; z.Es[4] = e11; z.Es[5] = e12;
    z.Es[6] = e02; z.Es[7] = e12; z.Es[8] = e22;
    z.k1 = ld(); z.k2 = ld(); z.k3 = ld();
  } else if (svk_fields(KIND)) {
    z.k1 = prm[0];
    z.k2 = prm[1];
#pragma unroll
    for (int i = 0; i < 9; ++i) z.Ci[i] = z.Pe[i] = T(0);  // not used by the SVK stress
  } else if (KIND == MAT_YEOH) {
    z.k1 = ld(); z.k2 = ld();
  }
}

// P += c * P_lin(G; frozen)
template <typename T, int KIND>
__device__ __forceinline__ void plin_add(const Frozen<T>& z, const T* G, T c, T* P) {
  if constexpr (KIND == MAT_SVK_TANGENT) {
    // dP = G S* + F* dS with S* = lambda tr(E*) I + 2 mu E*, E* = (F*^T F* - I) / 2,
    // dS = lambda tr(dE) I + 2 mu dE, dE = sym(F*^T G): the derivative of P(F) = F S(E(F))
    T Es[9], dE[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Es[3 * i + j] = T(0.5) * (z.F[i] * z.F[j] + z.F[3 + i] * z.F[3 + j] + z.F[6 + i] * z.F[6 + j] -
                                  ((i == j) ? T(1) : T(0)));
        dE[3 * i + j] = T(0.5) * (z.F[i] * G[j] + z.F[3 + i] * G[3 + j] + z.F[6 + i] * G[6 + j] +
                                  z.F[j] * G[i] + z.F[3 + j] * G[3 + i] + z.F[6 + j] * G[6 + i]);
      }
    const T ts = z.k1 * tr3(Es), td = z.k1 * tr3(dE);
    T Ss[9], dS[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      Ss[i] = T(2) * z.k2 * Es[i] + ((i % 4 == 0) ? ts : T(0));
      dS[i] = T(2) * z.k2 * dE[i] + ((i % 4 == 0) ? td : T(0));
    }
    T GS[9], FdS[9];
    matmul3(G, Ss, GS);
    matmul3(z.F, dS, FdS);
#pragma unroll
    for (int i = 0; i < 9; ++i) P[i] += c * (GS[i] + FdS[i]);
    return;
  }
  // E_lin = sym(G) + sym(D*^T G) / 2
  T DtG[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      DtG[3 * i + j] = z.Ds[i] * G[j] + z.Ds[3 + i] * G[3 + j] + z.Ds[6 + i] * G[6 + j];
  T El[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      El[3 * i + j] = T(0.5) * (G[3 * i + j] + G[3 * j + i]) +
                      T(0.25) * (DtG[3 * i + j] + DtG[3 * j + i]);
  T jl = T(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) jl += z.Pe[i] * G[i];
  T S[9];
  if (KIND == MAT_SVK) {
    const T t = z.k1 * tr3(El);
#pragma unroll
    for (int i = 0; i < 9; ++i) S[i] = T(2) * z.k2 * El[i] + ((i % 4 == 0) ? t : T(0));
  } else if (KIND == MAT_NEOHOOKE) {
    // S = 2 mu sym(Ci El) + lambda l* j_lin Ci
    T CE[9];
    matmul3(z.Ci, El, CE);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        S[3 * i + j] = T(0.5) * z.k1 * (CE[3 * i + j] + CE[3 * j + i]) + z.k2 * jl * z.Ci[3 * i + j];
  } else if (KIND == MAT_YEOH) {
    // S = alpha sym(Ci dev(2 El)) + beta j_lin Ci
    T dv[9];
    const T t = T(2) * tr3(El) / T(3);
#pragma unroll
    for (int i = 0; i < 9; ++i) dv[i] = T(2) * El[i] - ((i % 4 == 0) ? t : T(0));
    T CD[9];
    matmul3(z.Ci, dv, CD);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        S[3 * i + j] = T(0.5) * z.k1 * (CD[3 * i + j] + CD[3 * j + i]) + z.k2 * jl * z.Ci[3 * i + j];
  } else {  // MAT_MOONEY_RIVLIN
    const T es = tr3(z.Es), el = tr3(El);
    T ddot = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) ddot += z.Es[i] * El[i];
    T dv[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) dv[i] = T(2) * El[i] - ((i % 4 == 0) ? T(2) * el / T(3) : T(0));
    // E* E_lin + E_lin E* = X + X^T with X = E* E_lin (both symmetric)
    T X[9];
    matmul3(z.Es, El, X);
    // Q and dev(2 E_lin) are symmetric, so sym(Q C*^-1) = sym(C*^-1 Q) and the two
    // deviatoric terms share one product: sym(C*^-1 (k1 dev(2E_lin) + k2 Q))
    T Mq[9];
    const T iso = T(4) / T(3) * (es * el - ddot);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int a = 3 * i + j;
        const T q = dv[a] + T(2) * (es * El[a] + el * z.Es[a]) - T(2) * (X[a] + X[3 * j + i]) -
                    ((i == j) ? iso : T(0));
        Mq[a] = z.k1 * dv[a] + z.k2 * q;
      }
    T CM[9];
    matmul3(z.Ci, Mq, CM);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        S[3 * i + j] = T(0.5) * (CM[3 * i + j] + CM[3 * j + i]) + z.k3 * jl * z.Ci[3 * i + j];
  }
  T FS[9];
  matmul3(z.F, S, FS);
#pragma unroll
  for (int i = 0; i < 9; ++i) P[i] += c * FS[i];
}

// Small-strain stress lambda tr(eps) I + 2 mu eps, eps = sym(G); prm = {E, nu}.
template <typename T>
__device__ __forceinline__ void linear_stress(const T* prm, const T* G, T* P) {
  const T E = prm[0], nu = prm[1];
  const T lam = E * nu / ((T(1) + nu) * (T(1) - T(2) * nu));
  const T mu = E / (T(2) * (T(1) + nu));
  const T t = lam * tr3(G);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      P[3 * i + j] = mu * (G[3 * i + j] + G[3 * j + i]) + (i == j ? t : T(0));
}

// Strain energy density psi(F) (FP64), F = I + D.
__device__ __forceinline__ double psi_of(int kind, const double* prm, const double* D) {
  if (kind == MAT_LINEAR) {
    const double E = prm[0], nu = prm[1];
    const double lam = E * nu / ((1 + nu) * (1 - 2 * nu)), mu = E / (2 * (1 + nu));
    double tr = D[0] + D[4] + D[8], ee = 0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const double e = 0.5 * (D[3 * i + j] + D[3 * j + i]);
        ee += e * e;
      }
    return 0.5 * lam * tr * tr + mu * ee;
  }
  double F[9];
  for (int i = 0; i < 9; ++i) F[i] = D[i] + ((i % 4 == 0) ? 1.0 : 0.0);
  double C[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  const double J = det3(F);
  const double I1 = C[0] + C[4] + C[8];
  double CC = 0;
  for (int i = 0; i < 9; ++i) CC += C[i] * C[i];  // tr(C^2), C symmetric
  if (kind == MAT_NEOHOOKE) {
    const double lnJ = log(J);
    return 0.5 * prm[0] * (I1 - 3) - prm[0] * lnJ + 0.5 * prm[1] * lnJ * lnJ;
  }
  if (kind == MAT_MOONEY_RIVLIN) {
    const double I2 = 0.5 * (I1 * I1 - CC);
    const double a = 1.0 / (cbrt(J) * cbrt(J));
    return prm[0] * (a * I1 - 3) + prm[1] * (a * a * I2 - 3) + 0.5 * prm[2] * (J - 1) * (J - 1);
  }
  if (kind == MAT_SVK) {
    double E[9];
    for (int i = 0; i < 9; ++i) E[i] = 0.5 * (C[i] - ((i % 4 == 0) ? 1.0 : 0.0));
    double trE = E[0] + E[4] + E[8], EE = 0;
    for (int i = 0; i < 9; ++i) EE += E[i] * E[i];
    return 0.5 * prm[0] * trE * trE + prm[1] * EE;
  }
  // Yeoh
  const double a = 1.0 / (cbrt(J) * cbrt(J));
  const double x = a * I1 - 3;
  return prm[0] * x + prm[1] * x * x + prm[2] * x * x * x + (J - 1) * (J - 1) / prm[3];
}

}  // namespace etp
