// Per-tetrahedron element math for the tet maps (device code).
//
// Linear tetrahedra (the element of Ebb's FEM tetmesh domain, Section 5.2;
// StVK per Section 7.2, neo-Hookean per Section 7.3; the paper prints no
// formulas, these are the textbook ones).  All matrices are 3x3 row-major
// arrays.  Everything is written in terms of the displacement gradient
//     G = Du B = F - I,   Du = [u1-u0, u2-u0, u3-u0],   B = Dm^-1
// so that small strains are formed without the cancellation of F^T F - I or
// F - F^-T; that keeps FP32 results relatively accurate at small strain.
//
//   StVK: E = (G + G^T + G^T G)/2, S = 2 mu E + lam tr(E) I, P = S + G S
//         dE = sym(dF + G^T dF),  dP = dF S + (I + G)(2 mu dE + lam tr(dE) I)
//   NH:   J - 1 = tr G + ((tr G)^2 - tr(G^2))/2 + det G,  ln J = log1p(J - 1)
//         F^-T = cof(F) / J,  F - F^-T = G + G^T F^-T
//         P  = mu (G + G^T F^-T) + lam ln J F^-T
//         dP = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam (F^-T : dF) F^-T
//
// diag(K) per corner a and component c has a closed form because the probe
// dF = e_c b^T is rank one (b = row a-1 of B for a = 1..3, b_0 = -sum):
//   NH:   V (mu |b|^2 + (mu + lam - lam ln J) g_c^2),  g = F^-T b
//   StVK: V (b^T S b + mu (|q|^2 |b|^2 + (q.b)^2) + lam (q.b)^2),  q = row c of F
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace ebb {

template <typename T> __device__ __forceinline__ T ebb_log1p(T x);
template <> __device__ __forceinline__ float ebb_log1p<float>(float x) { return log1pf(x); }
template <> __device__ __forceinline__ double ebb_log1p<double>(double x) { return log1p(x); }

// C = A * B
template <typename T>
__device__ __forceinline__ void mm(const T* A, const T* B, T* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[i * 3 + j] = A[i * 3 + 0] * B[0 * 3 + j] + A[i * 3 + 1] * B[1 * 3 + j] + A[i * 3 + 2] * B[2 * 3 + j];
}

// C = A^T * B
template <typename T>
__device__ __forceinline__ void mtm(const T* A, const T* B, T* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[i * 3 + j] = A[0 * 3 + i] * B[0 * 3 + j] + A[1 * 3 + i] * B[1 * 3 + j] + A[2 * 3 + i] * B[2 * 3 + j];
}

// ---------------------------------------------------------------- StVK ----
template <typename T>
struct StvkState {
  T G[9];  // F - I
  T S[9];  // second Piola-Kirchhoff stress
};

template <typename T>
__device__ __forceinline__ void stvk_state(const T* G, T mu, T lam, StvkState<T>& st) {
#pragma unroll
  for (int i = 0; i < 9; ++i) st.G[i] = G[i];
  T GtG[9];
  mtm(G, G, GtG);
  T E[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) E[i * 3 + j] = T(0.5) * (G[i * 3 + j] + G[j * 3 + i] + GtG[i * 3 + j]);
  const T trE = E[0] + E[4] + E[8];
#pragma unroll
  for (int i = 0; i < 9; ++i) st.S[i] = T(2) * mu * E[i];
  st.S[0] += lam * trE;
  st.S[4] += lam * trE;
  st.S[8] += lam * trE;
}

// P = F S = S + G S
template <typename T>
__device__ __forceinline__ void stvk_P(const StvkState<T>& st, T* P) {
  mm(st.G, st.S, P);
#pragma unroll
  for (int i = 0; i < 9; ++i) P[i] += st.S[i];
}

template <typename T>
__device__ __forceinline__ void stvk_dP(const StvkState<T>& st, T mu, T lam, const T* dF, T* dP) {
  // W = F^T dF = dF + G^T dF ; dE = sym(W)
  T W[9];
  mtm(st.G, dF, W);
#pragma unroll
  for (int i = 0; i < 9; ++i) W[i] += dF[i];
  const T trdE = W[0] + W[4] + W[8];
  T Y[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Y[i * 3 + j] = mu * (W[i * 3 + j] + W[j * 3 + i]);
  Y[0] += lam * trdE;
  Y[4] += lam * trdE;
  Y[8] += lam * trdE;
  // dP = dF S + Y + G Y
  T A[9], C[9];
  mm(dF, st.S, A);
  mm(st.G, Y, C);
#pragma unroll
  for (int i = 0; i < 9; ++i) dP[i] = A[i] + Y[i] + C[i];
}

// diag entries of corner with gradient row b, for components c = 0..2 (times V outside)
template <typename T>
__device__ __forceinline__ void stvk_diag(const StvkState<T>& st, T mu, T lam, const T* b, T* out) {
  const T bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  T Sb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Sb[i] = st.S[i * 3 + 0] * b[0] + st.S[i * 3 + 1] * b[1] + st.S[i * 3 + 2] * b[2];
  const T bSb = b[0] * Sb[0] + b[1] * Sb[1] + b[2] * Sb[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    // q = row c of F = e_c + row c of G
    T q0 = st.G[c * 3 + 0], q1 = st.G[c * 3 + 1], q2 = st.G[c * 3 + 2];
    if (c == 0) q0 += T(1);
    if (c == 1) q1 += T(1);
    if (c == 2) q2 += T(1);
    const T qq = q0 * q0 + q1 * q1 + q2 * q2;
    const T qb = q0 * b[0] + q1 * b[1] + q2 * b[2];
    out[c] = bSb + mu * (qq * bb + qb * qb) + lam * qb * qb;
  }
}

// ---------------------------------------------------------- neo-Hookean ----
template <typename T>
struct NhState {
  T G[9];
  T FiT[9];  // F^-T
  T lnJ;
};

// Returns false if J <= 0 (inverted element).
template <typename T>
__device__ __forceinline__ bool nh_state(const T* G, NhState<T>& st) {
#pragma unroll
  for (int i = 0; i < 9; ++i) st.G[i] = G[i];
  const T trG = G[0] + G[4] + G[8];
  const T trG2 = G[0] * G[0] + G[4] * G[4] + G[8] * G[8] +
                 T(2) * (G[1] * G[3] + G[2] * G[6] + G[5] * G[7]);
  const T detG = G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                 G[2] * (G[3] * G[7] - G[4] * G[6]);
  const T Jm1 = trG + T(0.5) * (trG * trG - trG2) + detG;
  const T J = T(1) + Jm1;
  if (!(J > T(0))) return false;
  st.lnJ = ebb_log1p(Jm1);
  const T F0 = T(1) + G[0], F1 = G[1], F2 = G[2];
  const T F3 = G[3], F4 = T(1) + G[4], F5 = G[5];
  const T F6 = G[6], F7 = G[7], F8 = T(1) + G[8];
  const T iJ = T(1) / J;
  st.FiT[0] = (F4 * F8 - F5 * F7) * iJ;
  st.FiT[1] = (F5 * F6 - F3 * F8) * iJ;
  st.FiT[2] = (F3 * F7 - F4 * F6) * iJ;
  st.FiT[3] = (F2 * F7 - F1 * F8) * iJ;
  st.FiT[4] = (F0 * F8 - F2 * F6) * iJ;
  st.FiT[5] = (F1 * F6 - F0 * F7) * iJ;
  st.FiT[6] = (F1 * F5 - F2 * F4) * iJ;
  st.FiT[7] = (F2 * F3 - F0 * F5) * iJ;
  st.FiT[8] = (F0 * F4 - F1 * F3) * iJ;
  return true;
}

// P = mu (G + G^T F^-T) + lam ln J F^-T
template <typename T>
__device__ __forceinline__ void nh_P(const NhState<T>& st, T mu, T lam, T* P) {
  T GtFiT[9];
  mtm(st.G, st.FiT, GtFiT);
  const T ll = lam * st.lnJ;
#pragma unroll
  for (int i = 0; i < 9; ++i) P[i] = mu * (st.G[i] + GtFiT[i]) + ll * st.FiT[i];
}

template <typename T>
__device__ __forceinline__ void nh_dP(const NhState<T>& st, T mu, T lam, const T* dF, T* dP) {
  // T1 = dF^T F^-T ; A = F^-T T1 = F^-T dF^T F^-T
  T T1[9], A[9];
  mtm(dF, st.FiT, T1);
  mm(st.FiT, T1, A);
  T tr = T(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) tr += st.FiT[i] * dF[i];
  const T c1 = mu - lam * st.lnJ;
  const T c2 = lam * tr;
#pragma unroll
  for (int i = 0; i < 9; ++i) dP[i] = mu * dF[i] + c1 * A[i] + c2 * st.FiT[i];
}

template <typename T>
__device__ __forceinline__ void nh_diag(const NhState<T>& st, T mu, T lam, const T* b, T* out) {
  const T bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const T c = mu + lam - lam * st.lnJ;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T g = st.FiT[i * 3 + 0] * b[0] + st.FiT[i * 3 + 1] * b[1] + st.FiT[i * 3 + 2] * b[2];
    out[i] = mu * bb + c * g * g;
  }
}

}  // namespace ebb
