// Cooperative element map (device code): three lanes per tet.
//
// Section 8 names "several threads per row" among the schedules the paper's
// one-row-per-thread GPU backend leaves out.  Here lane r of a group of three
// computes row r of every per-tet matrix the element forms -- row r of
// G = Du Dm^-1 from component r of the corner displacements, row r of P and
// dP, and component r of each corner's force, K w and diag(K) -- and the
// rows a lane needs from its neighbours (G, dF and the symmetric-part
// matrices) come through warp shuffles.  The formulas are those of
// tet_math.cuh (Section 7.2 StVK, Section 7.3 neo-Hookean, written with
// G = F - I), split by row; the neo-Hookean state (J, ln J, F^-T) is formed
// from the gathered G in every lane of the group, identically.  A warp holds
// ten groups (lanes 30 and 31 only take part in the shuffles); each lane adds
// its component of every corner output with one atomic.
#pragma once

#include "ebb_internal.h"
#include "tet_io.cuh"
#include "tet_math.cuh"

namespace ebb {

constexpr int kCoopThreads = 128;
constexpr int kCoopTetsPerWarp = 10;
constexpr int kCoopTetsPerBlock = kCoopTetsPerWarp * (kCoopThreads / 32);

template <typename T>
__device__ __forceinline__ T grp_shfl(T v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// full[3c + j] = row[j] of lane base + c.
template <typename T>
__device__ __forceinline__ void gather_rows(const T (&row)[3], T (&full)[9], int base) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int j = 0; j < 3; ++j) full[3 * c + j] = grp_shfl(row[j], base + c);
}

// Sum of v over the group's three lanes (every lane gets the same sum, added
// in lane order).
template <typename T>
__device__ __forceinline__ T group_sum(T v, int base) {
  const T a = grp_shfl(v, base), b = grp_shfl(v, base + 1), c = grp_shfl(v, base + 2);
  return (a + b) + c;
}

// Row or column r of a 3x3 row-major matrix, picked by selects rather than
// a run-time index (which would move the matrix to local memory).
template <typename T>
__device__ __forceinline__ T sel3(int r, T a, T b, T c) {
  return r == 0 ? a : (r == 1 ? b : c);
}
template <typename T>
__device__ __forceinline__ void row_of(const T (&M)[9], int r, T (&out)[3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j) out[j] = sel3(r, M[j], M[3 + j], M[6 + j]);
}
template <typename T>
__device__ __forceinline__ void col_of(const T (&M)[9], int r, T (&out)[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = sel3(r, M[3 * i], M[3 * i + 1], M[3 * i + 2]);
}

// Component r of the four corner outputs from row r of a stress-like matrix
// X: out[a] = s V (X_r . b_a) for a = 1..3 (b_a = row a-1 of B), corner 0
// minus their sum.
template <typename T>
__device__ __forceinline__ void coop_corners(const T (&Xr)[3], const T* B, T sV, T (&out)[4]) {
  T s0 = T(0);
#pragma unroll
  for (int a = 1; a <= 3; ++a) {
    out[a] = sV * (Xr[0] * B[(a - 1) * 3 + 0] + Xr[1] * B[(a - 1) * 3 + 1] + Xr[2] * B[(a - 1) * 3 + 2]);
    s0 -= out[a];
  }
  out[0] = s0;
}

template <typename T, int MODEL, int OPS, bool AOS>
__global__ void __launch_bounds__(kCoopThreads)
tet_coop_kernel(int nt, int nv, const int4* __restrict__ keys, const int* __restrict__ perm, TetStreams<T> s,
                T mu0, T lam0, MapIO<T> io, const int* active, int* err) {
  if (active != nullptr && *active == 0) return;
  const int lane = threadIdx.x & 31;
  const int grp = lane / 3;
  const int r = lane - 3 * grp;            // the row this lane computes
  const int base = 3 * grp;                // first lane of the group
  const int t = (blockIdx.x * (kCoopThreads / 32) + (threadIdx.x >> 5)) * kCoopTetsPerWarp + grp;
  const bool act = grp < kCoopTetsPerWarp && t < nt;
  const int tc = act ? t : 0;              // lanes without a tet work on tet 0 and discard it
  const int4 k4 = keys[tc];
  const int kk[4] = {k4.x, k4.y, k4.z, k4.w};
  T B[9], V, mu, lam;
  load_tet(s, nt, tc, mu0, lam0, B, V, mu, lam);
  const int rc = r < 3 ? r : 0;
  auto comp = [&](const T* f, int v) -> T {
    return AOS ? f[4 * (size_t)v + rc] : f[(size_t)rc * nv + v];
  };
  // row r of Du and of G = Du B (and of Dw, dF = Dw B)
  T Gr[3], dFr[3] = {T(0), T(0), T(0)};
  {
    const T u0 = comp(io.u, kk[0]);
    T Du[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) Du[j] = comp(io.u, kk[j + 1]) - u0;
#pragma unroll
    for (int j = 0; j < 3; ++j) Gr[j] = Du[0] * B[0 * 3 + j] + Du[1] * B[1 * 3 + j] + Du[2] * B[2 * 3 + j];
    if (OPS & OP_KV) {
      const T w0 = comp(io.w, kk[0]);
      T Dw[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) Dw[j] = comp(io.w, kk[j + 1]) - w0;
#pragma unroll
      for (int j = 0; j < 3; ++j) dFr[j] = Dw[0] * B[0 * 3 + j] + Dw[1] * B[1 * 3 + j] + Dw[2] * B[2 * 3 + j];
    }
  }
  T G[9];
  gather_rows(Gr, G, base);
  T dF[9];
  if (OPS & OP_KV) gather_rows(dFr, dF, base);
  T Gc[3];                                 // column r of G
  col_of(G, rc, Gc);

  T fo[4] = {T(0), T(0), T(0), T(0)}, ko[4] = {T(0), T(0), T(0), T(0)}, dgo[4] = {T(0), T(0), T(0), T(0)};
  bool good = true;
  if (MODEL == EBB_STVK) {
    // E row r = (G_r + G^T_r + (G^T G)_r) / 2, gathered; S = 2 mu E + lam tr(E) I
    T Er[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Er[j] = T(0.5) * (Gr[j] + Gc[j] + (Gc[0] * G[0 * 3 + j] + Gc[1] * G[1 * 3 + j] + Gc[2] * G[2 * 3 + j]));
    T S[9];
    gather_rows(Er, S, base);
    const T trE = S[0] + S[4] + S[8];
#pragma unroll
    for (int i = 0; i < 9; ++i) S[i] = T(2) * mu * S[i];
    S[0] += lam * trE;
    S[4] += lam * trE;
    S[8] += lam * trE;
    T Sr[3];
    row_of(S, rc, Sr);
    if (OPS & OP_FORCE) {
      // P row r = S_r + G_r S
      T Pr[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) Pr[j] = Sr[j] + Gr[0] * S[0 * 3 + j] + Gr[1] * S[1 * 3 + j] + Gr[2] * S[2 * 3 + j];
      coop_corners(Pr, B, -V, fo);
    }
    if (OPS & OP_KV) {
      // W row r = dF_r + (G^T dF)_r, gathered; Y = mu (W + W^T) + lam tr(W) I
      T Wr[3];
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Wr[j] = dFr[j] + Gc[0] * dF[0 * 3 + j] + Gc[1] * dF[1 * 3 + j] + Gc[2] * dF[2 * 3 + j];
      T W[9];
      gather_rows(Wr, W, base);
      const T trW = W[0] + W[4] + W[8];
      T Y[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Y[i * 3 + j] = mu * (W[i * 3 + j] + W[j * 3 + i]);
      Y[0] += lam * trW;
      Y[4] += lam * trW;
      Y[8] += lam * trW;
      T Yr[3];
      row_of(Y, rc, Yr);
      // dP row r = dF_r S + Y_r + G_r Y
      T dPr[3];
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dPr[j] = dFr[0] * S[0 * 3 + j] + dFr[1] * S[1 * 3 + j] + dFr[2] * S[2 * 3 + j] + Yr[j] +
                 Gr[0] * Y[0 * 3 + j] + Gr[1] * Y[1 * 3 + j] + Gr[2] * Y[2 * 3 + j];
      coop_corners(dPr, B, V, ko);
    }
    if (OPS & OP_DIAG) {
      // q = row r of F; per corner b: V (b^T S b + mu (|q|^2 |b|^2 + (q.b)^2) + lam (q.b)^2)
      const T q[3] = {Gr[0] + (rc == 0 ? T(1) : T(0)), Gr[1] + (rc == 1 ? T(1) : T(0)),
                      Gr[2] + (rc == 2 ? T(1) : T(0))};
      const T qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        T b[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) b[j] = a == 0 ? -(B[j] + B[3 + j] + B[6 + j]) : B[(a - 1) * 3 + j];
        const T bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        T bSb = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) bSb += b[i] * (S[i * 3 + 0] * b[0] + S[i * 3 + 1] * b[1] + S[i * 3 + 2] * b[2]);
        const T qb = q[0] * b[0] + q[1] * b[1] + q[2] * b[2];
        dgo[a] = V * (bSb + mu * (qq * bb + qb * qb) + lam * qb * qb);
      }
    }
  } else {
    // The same full G in every lane of the group: the same J, ln J, F^-T.
    // Every lane runs the shuffles below whatever its tet's J (an inverted
    // tet's values are discarded), so that no shuffle misses a lane.
    NhState<T> sn{};
    good = nh_state(G, sn);
    T Fr[3];                               // row r of F^-T
    row_of(sn.FiT, rc, Fr);
    {
      if (OPS & OP_FORCE) {
        // P row r = mu (G_r + (G^T F^-T)_r) + lam ln J F^-T_r
        const T ll = lam * sn.lnJ;
        T Pr[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          Pr[j] = mu * (Gr[j] + (Gc[0] * sn.FiT[0 * 3 + j] + Gc[1] * sn.FiT[1 * 3 + j] + Gc[2] * sn.FiT[2 * 3 + j])) +
                  ll * Fr[j];
        coop_corners(Pr, B, -V, fo);
      }
      if (OPS & OP_KV) {
        // T1 row r = (dF^T F^-T)_r, gathered; dP row r = mu dF_r + (mu - lam ln J) (F^-T T1)_r
        // + lam tr(F^-1 dF) F^-T_r
        T dFc[3];                          // column r of dF
        col_of(dF, rc, dFc);
        T T1r[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          T1r[j] = dFc[0] * sn.FiT[0 * 3 + j] + dFc[1] * sn.FiT[1 * 3 + j] + dFc[2] * sn.FiT[2 * 3 + j];
        T T1[9];
        gather_rows(T1r, T1, base);
        const T tr = group_sum(Fr[0] * dFr[0] + Fr[1] * dFr[1] + Fr[2] * dFr[2], base);
        const T c1 = mu - lam * sn.lnJ;
        const T c2 = lam * tr;
        T dPr[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
          dPr[j] = mu * dFr[j] + c1 * (Fr[0] * T1[0 * 3 + j] + Fr[1] * T1[1 * 3 + j] + Fr[2] * T1[2 * 3 + j]) +
                   c2 * Fr[j];
        coop_corners(dPr, B, V, ko);
      }
      if (OPS & OP_DIAG) {
        // per corner b: V (mu |b|^2 + (mu + lam - lam ln J) g_r^2), g = F^-T b
        const T c = mu + lam - lam * sn.lnJ;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T b[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) b[j] = a == 0 ? -(B[j] + B[3 + j] + B[6 + j]) : B[(a - 1) * 3 + j];
          const T bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
          const T g = Fr[0] * b[0] + Fr[1] * b[1] + Fr[2] * b[2];
          dgo[a] = V * (mu * bb + c * g * g);
        }
      }
    }
    if (!good && act && r == 0) raise_error(err, EBB_ERR_INVERTED, perm[t]);
  }
  if (!act || !good) return;
  // component r of every corner output, one atomic each
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const size_t o = AOS ? 4 * (size_t)kk[a] + rc : (size_t)rc * nv + kk[a];
    if (OPS & OP_FORCE) atomicAdd(io.f + o, fo[a]);
    if (OPS & OP_KV) atomicAdd(io.Kw + o, ko[a]);
    if (OPS & OP_DIAG) atomicAdd(io.d + o, dgo[a]);
  }
}

}  // namespace ebb
