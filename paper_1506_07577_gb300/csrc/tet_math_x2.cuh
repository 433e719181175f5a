// Paired FP32 element math for the maps that compute K w (device code,
// sm_100+ paired FP32 instructions).
//
// Each matrix the K w path forms has a twin of the same shape on the force
// path, built from the same shared operand:
//     G = Du B           beside  dF = Dw B
//     G^T G              beside  G^T dF            (StVK)
//     G S                beside  dF S              (StVK)
//     G^T F^-T           beside  dF^T F^-T         (neo-Hookean)
//     P                  beside  dP
//     -V P b_a           beside  V dP b_a          (corner outputs)
// Holding the twins as the two lanes of a float2, one paired instruction
// (__ffma2_rn / __fmul2_rn / __fadd2_rn) forms both, the shared operand
// broadcast to both lanes.  Lane x is the force path, lane y the K w path.
// The formulas are those of tet_math.cuh (Sections 7.2 and 7.3 models,
// written in terms of G = F - I); only the association of some sums differs.
#pragma once

#include <cuda_runtime.h>

#include "tet_math.cuh"

namespace ebb {

__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }

// C = X S, S shared: C[i][j] = sum_k X[i][k] S[k][j]
__device__ __forceinline__ void mm_x2(const float2* X, const float* S, float2* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float2 s = __fmul2_rn(X[i * 3 + 0], bc2(S[0 * 3 + j]));
      s = __ffma2_rn(X[i * 3 + 1], bc2(S[1 * 3 + j]), s);
      C[i * 3 + j] = __ffma2_rn(X[i * 3 + 2], bc2(S[2 * 3 + j]), s);
    }
}

// C = X^T S, S shared: C[i][j] = sum_k X[k][i] S[k][j]
__device__ __forceinline__ void mtm_x2(const float2* X, const float* S, float2* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float2 s = __fmul2_rn(X[0 * 3 + i], bc2(S[0 * 3 + j]));
      s = __ffma2_rn(X[1 * 3 + i], bc2(S[1 * 3 + j]), s);
      C[i * 3 + j] = __ffma2_rn(X[2 * 3 + i], bc2(S[2 * 3 + j]), s);
    }
}

// C = S^T X, S shared: C[i][j] = sum_k S[k][i] X[k][j]
__device__ __forceinline__ void tmm_x2(const float* S, const float2* X, float2* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float2 s = __fmul2_rn(bc2(S[0 * 3 + i]), X[0 * 3 + j]);
      s = __ffma2_rn(bc2(S[1 * 3 + i]), X[1 * 3 + j], s);
      C[i * 3 + j] = __ffma2_rn(bc2(S[2 * 3 + i]), X[2 * 3 + j], s);
    }
}

// Corner outputs of the stress pair PP = (P, dP): lane x -V P b_a, lane y
// V dP b_a for a = 1..3 (b_a = row a-1 of B), corner 0 minus their sum.
__device__ __forceinline__ void corner_outputs_x2(const float2* PP, const float* B, float V, float2 (&out)[4][3]) {
  float2 Q[9];
  const float2 s = make_float2(-V, V);
#pragma unroll
  for (int i = 0; i < 9; ++i) Q[i] = __fmul2_rn(s, PP[i]);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int a = 1; a <= 3; ++a) {
      float2 t = __fmul2_rn(Q[c * 3 + 0], bc2(B[(a - 1) * 3 + 0]));
      t = __ffma2_rn(Q[c * 3 + 1], bc2(B[(a - 1) * 3 + 1]), t);
      out[a][c] = __ffma2_rn(Q[c * 3 + 2], bc2(B[(a - 1) * 3 + 2]), t);
    }
    out[0][c] = __fmul2_rn(bc2(-1.f), __fadd2_rn(__fadd2_rn(out[1][c], out[2][c]), out[3][c]));
  }
}

// StVK pair: S = 2 mu E + lam tr(E) I with E = (G + G^T + G^T G)/2;
// P = S + G S;  dP = dF S + Y + G Y with Y = 2 mu dE + lam tr(dE) I,
// 2 dE = W + W^T, W = dF + G^T dF.
__device__ __forceinline__ void stvk_eval_x2(const float* B, float V, float mu, float lam, const float2* D,
                                             float2 (&out)[4][3]) {
  float2 GD[9];
  mm_x2(D, B, GD);  // (G, dF)
  float G[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) G[i] = GD[i].x;
  float2 H[9];
  tmm_x2(G, GD, H);  // (G^T G, G^T dF)
#pragma unroll
  for (int i = 0; i < 9; ++i) H[i] = __fadd2_rn(H[i], GD[i]);  // (G + G^T G, W)
  float S[9], Y[9];
  const float trE = 0.5f * (H[0].x + G[0] + H[4].x + G[4] + H[8].x + G[8]);
  const float trdE = H[0].y + H[4].y + H[8].y;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      S[i * 3 + j] = mu * (H[i * 3 + j].x + G[j * 3 + i]);
      Y[i * 3 + j] = mu * (H[i * 3 + j].y + H[j * 3 + i].y);
    }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    S[i * 4] += lam * trE;
    Y[i * 4] += lam * trdE;
  }
  float2 GS[9];
  mm_x2(GD, S, GS);  // (G S, dF S)
  float C[9];
  mm(G, Y, C);
  float2 PP[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) PP[i] = __fadd2_rn(GS[i], make_float2(S[i], Y[i] + C[i]));
  corner_outputs_x2(PP, B, V, out);
}

// Neo-Hookean pair: P = mu (G + G^T F^-T) + lam ln J F^-T;
// dP = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam (F^-T : dF) F^-T.
// Returns false for an inverted element (J <= 0).
__device__ __forceinline__ bool nh_eval_x2(const float* B, float V, float mu, float lam, const float2* D,
                                           float2 (&out)[4][3]) {
  float2 GD[9];
  mm_x2(D, B, GD);  // (G, dF)
  float G[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) G[i] = GD[i].x;
  NhState<float> sn;
  if (!nh_state(G, sn)) return false;
  float2 T1[9];
  mtm_x2(GD, sn.FiT, T1);  // (G^T F^-T, dF^T F^-T)
  float T1y[9], A[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) T1y[i] = T1[i].y;
  mm(sn.FiT, T1y, A);  // F^-T dF^T F^-T
  float tr = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i) tr += sn.FiT[i] * GD[i].y;
  const float2 m2 = bc2(mu);
  const float2 c1 = make_float2(mu, mu - lam * sn.lnJ);
  const float2 c2 = make_float2(lam * sn.lnJ, lam * tr);
  float2 PP[9];
#pragma unroll
  for (int i = 0; i < 9; ++i)
    PP[i] = __ffma2_rn(m2, GD[i], __ffma2_rn(c1, make_float2(T1[i].x, A[i]), __fmul2_rn(c2, bc2(sn.FiT[i]))));
  corner_outputs_x2(PP, B, V, out);
  return true;
}

}  // namespace ebb
