// Per-tet loads shared by the element kernels (device code): the tet's
// rest-shape data from the per-tet streams and the edge differences of the
// vertex fields it reads through its keys (tets.v, Section 5.2), and the
// device status word.
#pragma once

#include <cstdint>

#include "ebb_internal.h"

namespace ebb {

// First device-side error wins; `index` is reported with it (a caller row).
__device__ __forceinline__ void raise_error(int* err, int code, int index) {
  if (atomicCAS(err + ERRW_CODE, 0, code) == 0) err[ERRW_INDEX] = index;
}

// Dm^-1 (B), rest volume and Lame parameters of internal tet t.
template <typename T>
__device__ __forceinline__ void load_tet(const TetStreams<T>& s, int nt, int t, T mu0, T lam0, T* B, T& V, T& mu,
                                         T& lam) {
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i] = s.B[(size_t)i * nt + t];
  V = s.V[t];
  mu = s.mu ? s.mu[t] : mu0;
  lam = s.lam ? s.lam[t] : lam0;
}

// Edge differences of u (and w) over one tet's corners kk: Du[c][j] =
// u_c(x_{j+1}) - u_c(x_0).  AOS: vertex-interleaved operands, one 16-byte
// load per corner and field.
template <typename T, int OPS, bool AOS>
__device__ __forceinline__ void load_edges(const MapIO<T>& io, int nv, const int (&kk)[4], T (&Du)[9], T (&Dw)[9]) {
  if constexpr (AOS) {
    float4 q[4], r[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      q[a] = reinterpret_cast<const float4*>(io.u)[kk[a]];
      if (OPS & OP_KV) r[a] = reinterpret_cast<const float4*>(io.w)[kk[a]];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Du[0 * 3 + j] = q[j + 1].x - q[0].x;
      Du[1 * 3 + j] = q[j + 1].y - q[0].y;
      Du[2 * 3 + j] = q[j + 1].z - q[0].z;
      if (OPS & OP_KV) {
        Dw[0 * 3 + j] = r[j + 1].x - r[0].x;
        Dw[1 * 3 + j] = r[j + 1].y - r[0].y;
        Dw[2 * 3 + j] = r[j + 1].z - r[0].z;
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* uc = io.u + (size_t)c * nv;
      const T u0 = uc[kk[0]];
#pragma unroll
      for (int j = 0; j < 3; ++j) Du[c * 3 + j] = uc[kk[j + 1]] - u0;
      if (OPS & OP_KV) {
        const T* wc = io.w + (size_t)c * nv;
        const T w0 = wc[kk[0]];
#pragma unroll
        for (int j = 0; j < 3; ++j) Dw[c * 3 + j] = wc[kk[j + 1]] - w0;
      }
    }
  }
}

}  // namespace ebb
