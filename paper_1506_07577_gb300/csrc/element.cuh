// Element evaluation shared by the map kernels (device code): force, K w
// and diag(K) of one tetrahedron from its rest data and edge differences.
#pragma once

#include "ebb_internal.h"
#include "tet_math.cuh"
#include "tet_math_x2.cuh"

namespace ebb {

// Evaluate one tet.  Du, Dw: edge differences [x1-x0, x2-x0, x3-x0] of the
// displacement and of the direction (3x3 row-major, row = component).  Outputs
// per corner a and component c: fo (force), ko (K w), dgo (diag K).
// Returns false for an inverted neo-Hookean element (J <= 0).
template <typename T, int MODEL, int OPS>
__device__ __forceinline__ bool element_eval(const T* B, T V, T mu, T lam, const T* Du, const T* Dw, T (&fo)[4][3],
                                             T (&ko)[4][3], T (&dgo)[4][3]) {
  if constexpr (sizeof(T) == 4 && OPS == (OP_FORCE | OP_KV)) {
    // FP32 force / K w pairs on the paired FP32 instructions (measured: the
    // K w map alone runs no faster paired, its force lane being idle work).
    float2 D[9], out[4][3];
#pragma unroll
    for (int i = 0; i < 9; ++i) D[i] = make_float2(Du[i], Dw[i]);
    if (MODEL == EBB_STVK)
      stvk_eval_x2(B, V, mu, lam, D, out);
    else if (!nh_eval_x2(B, V, mu, lam, D, out))
      return false;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fo[a][c] = out[a][c].x;
        ko[a][c] = out[a][c].y;
      }
    return true;
  }
  T G[9];
  mm(Du, B, G);
  StvkState<T> sv;
  NhState<T> sn;
  if (MODEL == EBB_STVK) {
    stvk_state(G, mu, lam, sv);
  } else {
    if (!nh_state(G, sn)) return false;
  }
  if (OPS & OP_FORCE) {
    T P[9];
    if (MODEL == EBB_STVK)
      stvk_P(sv, P);
    else
      nh_P(sn, mu, lam, P);
    // f_a = -V P b_a (b_a = row a-1 of B), f_0 = -sum
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T s0 = T(0);
#pragma unroll
      for (int a = 1; a <= 3; ++a) {
        const T val = -V * (P[c * 3 + 0] * B[(a - 1) * 3 + 0] + P[c * 3 + 1] * B[(a - 1) * 3 + 1] +
                            P[c * 3 + 2] * B[(a - 1) * 3 + 2]);
        fo[a][c] = val;
        s0 -= val;
      }
      fo[0][c] = s0;
    }
  }
  if (OPS & OP_KV) {
    T dF[9], dP[9];
    mm(Dw, B, dF);
    if (MODEL == EBB_STVK)
      stvk_dP(sv, mu, lam, dF, dP);
    else
      nh_dP(sn, mu, lam, dF, dP);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T s0 = T(0);
#pragma unroll
      for (int a = 1; a <= 3; ++a) {
        const T val = V * (dP[c * 3 + 0] * B[(a - 1) * 3 + 0] + dP[c * 3 + 1] * B[(a - 1) * 3 + 1] +
                           dP[c * 3 + 2] * B[(a - 1) * 3 + 2]);
        ko[a][c] = val;
        s0 -= val;
      }
      ko[0][c] = s0;
    }
  }
  if (OPS & OP_DIAG) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      T b[3];
      if (a == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) b[j] = -(B[j] + B[3 + j] + B[6 + j]);
      } else {
#pragma unroll
        for (int j = 0; j < 3; ++j) b[j] = B[(a - 1) * 3 + j];
      }
      T dg[3];
      if (MODEL == EBB_STVK)
        stvk_diag(sv, mu, lam, b, dg);
      else
        nh_diag(sn, mu, lam, b, dg);
#pragma unroll
      for (int c = 0; c < 3; ++c) dgo[a][c] = V * dg[c];
    }
  }
  return true;
}

}  // namespace ebb
