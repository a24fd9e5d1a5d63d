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
// The same for Neo-Hooke, Mooney-Rivlin and Yeoh: dP/dF[G] at the stored
// state by forward-mode differentiation of P(F) = F S(C) (dual numbers), on
// the stored coefficients of the material (only D* is used).
constexpr int MAT_NH_TANGENT = 6;
constexpr int MAT_MR_TANGENT = 7;
constexpr int MAT_YEOH_TANGENT = 8;
__host__ __device__ constexpr bool svk_fields(int kind) { return kind == MAT_SVK || kind == MAT_SVK_TANGENT; }
__host__ __device__ constexpr bool dual_tangent(int kind) {
  return kind == MAT_NH_TANGENT || kind == MAT_MR_TANGENT || kind == MAT_YEOH_TANGENT;
}
// Material whose stored coefficients a kind reads.
__host__ __device__ constexpr int base_material(int kind) {
  return kind == MAT_SVK_TANGENT ? MAT_SVK
         : kind == MAT_NH_TANGENT ? MAT_NEOHOOKE
         : kind == MAT_MR_TANGENT ? MAT_MOONEY_RIVLIN
         : kind == MAT_YEOH_TANGENT ? MAT_YEOH
                                    : kind;
}
// Internal tangent kind of a material for the Newton iterations of Newmark-beta.
inline int tangent_kind(int material) {
  switch (material) {
    case MAT_SVK: return MAT_SVK_TANGENT;
    case MAT_NEOHOOKE: return MAT_NH_TANGENT;
    case MAT_MOONEY_RIVLIN: return MAT_MR_TANGENT;
    case MAT_YEOH: return MAT_YEOH_TANGENT;
    default: return -1;
  }
}

// Dual number v + d eps (eps^2 = 0): one directional derivative alongside the value.
struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double r = a.v / b.v;
  return {r, (a.d - r * b.d) / b.v};
}
__device__ __forceinline__ Dual dlog(Dual a) { return {log(a.v), a.d / a.v}; }
// a^(-2/3)
__device__ __forceinline__ Dual dpow_m23(Dual a) {
  const double c = cbrt(a.v);
  const double r = 1.0 / (c * c);
  return {r, (-2.0 / 3.0) * r / a.v * a.d};
}

// First Piola stress P(F) = F S(C) of Neo-Hooke (prm = mu, lambda),
// Mooney-Rivlin (C10, C01, kappa) or Yeoh (C10, C20, C30, D1) in dual
// arithmetic (the laws of Section 2.1 and Appendix A.2):
//   NH:   S = mu (I - C^-1) + lambda ln J C^-1
//   MR:   S = 2 C10 J^-2/3 (I - I1/3 C^-1) + 2 C01 J^-4/3 (I1 I - C - 2 I2/3 C^-1) + kappa J (J - 1) C^-1
//   Yeoh: S = alpha (I - I1/3 C^-1) + 2/D1 J (J - 1) C^-1,
//         alpha = 2 J^-2/3 (C10 + 2 C20 (I1b - 3) + 3 C30 (I1b - 3)^2), I1b = J^-2/3 I1.
template <int BASE>
__device__ __forceinline__ void pk1_dual(const double* prm, const Dual* F, Dual* P) {
  Dual C[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = F[i] * F[j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  const Dual J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                 F[2] * (F[3] * F[7] - F[4] * F[6]);
  const Dual J2 = J * J;
  Dual Ci[9];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      Ci[3 * i + j] = (C[3 * i1 + j1] * C[3 * i2 + j2] - C[3 * i1 + j2] * C[3 * i2 + j1]) / J2;
    }
  }
  const Dual I1 = C[0] + C[4] + C[8];
  Dual S[9];
  if constexpr (BASE == MAT_NEOHOOKE) {
    const Dual lj = prm[1] * dlog(J);
#pragma unroll
    for (int k = 0; k < 9; ++k) S[k] = (k % 4 == 0 ? Dual{prm[0], 0.0} : Dual{0.0, 0.0}) - prm[0] * Ci[k] + lj * Ci[k];
  } else if constexpr (BASE == MAT_MOONEY_RIVLIN) {
    Dual CC{0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 9; ++k) CC = CC + C[k] * C[k];  // tr(C^2), C symmetric
    const Dual I2 = 0.5 * (I1 * I1 - CC);
    const Dual a = dpow_m23(J);
    const Dual a1 = (2.0 * prm[0]) * a, a2 = (2.0 * prm[1]) * (a * a);
    const Dual vol = prm[2] * (J * (J - Dual{1.0, 0.0}));
    const Dual t1 = (1.0 / 3.0) * I1, t2 = (2.0 / 3.0) * I2;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const Dual id = (k % 4 == 0) ? Dual{1.0, 0.0} : Dual{0.0, 0.0};
      S[k] = a1 * (id - t1 * Ci[k]) + a2 * (I1 * id - C[k] - t2 * Ci[k]) + vol * Ci[k];
    }
  } else {  // Yeoh
    const Dual a = dpow_m23(J);
    const Dual x = a * I1 - Dual{3.0, 0.0};
    const Dual alpha = 2.0 * (a * (Dual{prm[0], 0.0} + (2.0 * prm[1]) * x + (3.0 * prm[2]) * (x * x)));
    const Dual vol = (2.0 / prm[3]) * (J * (J - Dual{1.0, 0.0}));
    const Dual t1 = (1.0 / 3.0) * I1;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const Dual id = (k % 4 == 0) ? Dual{1.0, 0.0} : Dual{0.0, 0.0};
      S[k] = alpha * (id - t1 * Ci[k]) + vol * Ci[k];
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) P[3 * i + j] = F[3 * i] * S[j] + F[3 * i + 1] * S[3 + j] + F[3 * i + 2] * S[6 + j];
}

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
  T idet;   // 1 / J*^2
  T prm4[4];  // material parameters (dual tangents)
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
  z.idet = idet;
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
// state u* is fixed while the Arnoldi process runs, so grad u*, 1/J*^2 and the
// scalar material factors (which need cbrt or log) are evaluated once
// (k_frozen_build); every apply loads them and rebuilds F* = I + D*,
// C*^-1 = cof(C*) / J*^2, P_e(D*) and E* in registers (about a hundred
// multiply-adds per point, against streaming those 24 values from memory).
// Fields, each a separate plane of one value per (element, point):
//   D* (9); unless SVK: 1/J*^2; Neo-Hooke: k2; Mooney-Rivlin: k1, k2, k3;
//   Yeoh: k1, k2.
// Constant factors (2 mu for Neo-Hooke, lambda and mu for SVK) come from prm.
template <int KIND>
__host__ __device__ constexpr int frozen_nf() {
  return dual_tangent(KIND) ? frozen_nf<base_material(KIND)>()
         : KIND == MAT_LINEAR ? 0
         : svk_fields(KIND) ? 9
         : KIND == MAT_NEOHOOKE ? 11
         : KIND == MAT_MOONEY_RIVLIN ? 13
                                     : 12;  // Yeoh
}
inline int frozen_nf_of(int kind) {
  switch (kind) {
    case MAT_LINEAR: return frozen_nf<MAT_LINEAR>();
    case MAT_SVK: return frozen_nf<MAT_SVK>();
    case MAT_SVK_TANGENT: return frozen_nf<MAT_SVK_TANGENT>();
    case MAT_NEOHOOKE: return frozen_nf<MAT_NEOHOOKE>();
    case MAT_MOONEY_RIVLIN: return frozen_nf<MAT_MOONEY_RIVLIN>();
    case MAT_NH_TANGENT: return frozen_nf<MAT_NH_TANGENT>();
    case MAT_MR_TANGENT: return frozen_nf<MAT_MR_TANGENT>();
    case MAT_YEOH_TANGENT: return frozen_nf<MAT_YEOH_TANGENT>();
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
  if (!svk_fields(KIND)) v[f++] = z.idet;
  if (KIND == MAT_NEOHOOKE) v[f++] = z.k2;
  if (KIND == MAT_MOONEY_RIVLIN) { v[f++] = z.k1; v[f++] = z.k2; v[f++] = z.k3; }
  if (KIND == MAT_YEOH) { v[f++] = z.k1; v[f++] = z.k2; }
#pragma unroll
  for (int i = 0; i < NF; ++i) base[(int64_t)i * stride] = ok ? v[i] : T(0);
}

// Inverse of frozen_store: loads D*, 1/J*^2 and the scalar factors and
// rebuilds every field plin_add reads. A point stored as zeros (inverted at
// build time, already reported) gives F* = I and C*^-1 = 0.
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
  if constexpr (dual_tangent(KIND)) {  // the tangent rebuilds everything from F*
#pragma unroll
    for (int i = 0; i < 4; ++i) z.prm4[i] = prm[i];
    return;
  }
  T idet = T(0);
  if (!svk_fields(KIND)) idet = ld();
  if (KIND == MAT_NEOHOOKE) {
    z.k1 = T(2) * prm[0];
    z.k2 = ld();
  } else if (KIND == MAT_MOONEY_RIVLIN) {
    z.k1 = ld(); z.k2 = ld(); z.k3 = ld();
  } else if (KIND == MAT_YEOH) {
    z.k1 = ld(); z.k2 = ld();
  } else if (svk_fields(KIND)) {
    z.k1 = prm[0];
    z.k2 = prm[1];
  }
  if (!svk_fields(KIND) && KIND != MAT_LINEAR) {
    // C* = F*^T F* (symmetric), C*^-1 = cof(C*) / det(C*), det(C*) = J*^2
    T C[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        C[3 * i + j] = z.F[i] * z.F[j] + z.F[3 + i] * z.F[3 + j] + z.F[6 + i] * z.F[6 + j];
        C[3 * j + i] = C[3 * i + j];
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        const T c = (C[3 * i1 + j1] * C[3 * i2 + j2] - C[3 * i1 + j2] * C[3 * i2 + j1]) * idet;
        z.Ci[3 * i + j] = c;
        z.Ci[3 * j + i] = c;
      }
    T cD[9];
    cof3(z.Ds, cD);
    const T trD = tr3(z.Ds);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        z.Pe[3 * i + j] = (i == j ? T(1) + T(0.5) * trD : T(0)) - T(0.5) * z.Ds[3 * j + i] + cD[3 * i + j] * T(1.0 / 3.0);
    if (KIND == MAT_MOONEY_RIVLIN) {
#pragma unroll
      for (int i = 0; i < 9; ++i) z.Es[i] = T(0.5) * (C[i] - ((i % 4 == 0) ? T(1) : T(0)));
    }
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
  if constexpr (dual_tangent(KIND)) {
    // dP/dF[G] at F*: the eps-part of P(F* + eps G)
    Dual Fd[9], Pd[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Fd[i] = Dual{(double)z.F[i], (double)G[i]};
    double prm64[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) prm64[i] = (double)z.prm4[i];
    pk1_dual<base_material(KIND)>(prm64, Fd, Pd);
#pragma unroll
    for (int i = 0; i < 9; ++i) P[i] += c * (T)Pd[i].d;
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
