// Element maps over the tets relation: elastic force, K w and diag(K),
// reduced (+=) into vertex fields.
//
// A map is Ebb's kernel over a relation (Section 4.1): one instance per tet
// reads the tet's four vertex keys (tets.v[4], Section 5.2), gathers vertex
// fields through them and reduces per-corner results into vertex fields.
// Three reduction strategies share one element evaluation:
//   direct  one thread per tet, hardware atomic adds (Section 6.2
//           "Reductions"), or plain read-modify-write inside one colour of a
//           vertex-conflict colouring (Section 7.4, Liszt's colouring);
//   tiled   one CTA per tile of Morton-ordered tets: the tile's distinct
//           vertices are gathered into shared memory once, per-corner results
//           are pre-reduced there with shared-memory atomics, and each distinct
//           vertex gets one global atomic add per component.
#include <cstdint>

#include "ebb_internal.h"
#include "tet_math.cuh"

namespace ebb {

namespace {

constexpr int kMapThreads = 128;

__device__ __forceinline__ void raise_error(int* err, int code, int index) {
  if (atomicCAS(err + ERRW_CODE, 0, code) == 0) err[ERRW_INDEX] = index;
}

// Evaluate one tet.  Du, Dw: edge differences [x1-x0, x2-x0, x3-x0] of the
// displacement and of the direction (3x3 row-major, row = component).  Outputs
// per corner a and component c: fo (force), ko (K w), dgo (diag K).
// Returns false for an inverted neo-Hookean element (J <= 0).
template <typename T, int MODEL, int OPS>
__device__ __forceinline__ bool element_eval(const T* B, T V, T mu, T lam, const T* Du, const T* Dw, T (&fo)[4][3],
                                             T (&ko)[4][3], T (&dgo)[4][3]) {
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

template <typename T>
__device__ __forceinline__ void load_tet(const TetStreams<T>& s, int nt, int t, T mu0, T lam0, T* B, T& V, T& mu,
                                         T& lam) {
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i] = s.B[(size_t)i * nt + t];
  V = s.V[t];
  mu = s.mu ? s.mu[t] : mu0;
  lam = s.lam ? s.lam[t] : lam0;
}

// ---- direct: one thread per tet -------------------------------------------
template <typename T, int MODEL, int OPS, bool ATOMIC>
__global__ void __launch_bounds__(kMapThreads)
tet_map_kernel(int t_begin, int t_end, int nt, int nv, const int4* __restrict__ keys, const int* __restrict__ perm,
               TetStreams<T> s, T mu0, T lam0, MapIO<T> io, const int* active, int* err) {
  if (active != nullptr && *active == 0) return;
  const int t = t_begin + blockIdx.x * kMapThreads + threadIdx.x;
  if (t >= t_end) return;
  const int4 k4 = keys[t];
  const int kk[4] = {k4.x, k4.y, k4.z, k4.w};
  T B[9], V, mu, lam;
  load_tet(s, nt, t, mu0, lam0, B, V, mu, lam);
  T Du[9], Dw[9];
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
  T fo[4][3], ko[4][3], dgo[4][3];
  if (!element_eval<T, MODEL, OPS>(B, V, mu, lam, Du, Dw, fo, ko, dgo)) {
    raise_error(err, EBB_ERR_INVERTED, perm[t]);
    return;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * nv + kk[a];
      if (ATOMIC) {
        if (OPS & OP_FORCE) atomicAdd(io.f + o, fo[a][c]);
        if (OPS & OP_KV) atomicAdd(io.Kw + o, ko[a][c]);
        if (OPS & OP_DIAG) atomicAdd(io.d + o, dgo[a][c]);
      } else {
        if (OPS & OP_FORCE) io.f[o] += fo[a][c];
        if (OPS & OP_KV) io.Kw[o] += ko[a][c];
        if (OPS & OP_DIAG) io.d[o] += dgo[a][c];
      }
    }
  }
}

// ---- tiled: one CTA per tile, shared-memory gather and pre-reduction --------
template <typename T, int MODEL, int OPS>
__global__ void __launch_bounds__(kTileTets)
tet_tile_kernel(int nt, int nv, const int* __restrict__ tet_off, const int* __restrict__ vtx_off,
                const int* __restrict__ vtx, const uchar4* __restrict__ slots, const int* __restrict__ perm,
                TetStreams<T> s, T mu0, T lam0, MapIO<T> io, const int* active, int* err) {
  constexpr bool FO = (OPS & OP_FORCE) != 0;
  constexpr bool KV = (OPS & OP_KV) != 0;
  constexpr bool DG = (OPS & OP_DIAG) != 0;
  constexpr int S = kTileSlots;
  __shared__ T su[3][S];
  __shared__ T sw[KV ? 3 : 1][KV ? S : 1];
  __shared__ T sf[FO ? 3 : 1][FO ? S : 1];
  __shared__ T sk[KV ? 3 : 1][KV ? S : 1];
  __shared__ T sd[DG ? 3 : 1][DG ? S : 1];
  __shared__ int sid[S];
  if (active != nullptr && *active == 0) return;
  const int tile = blockIdx.x;
  const int tb = tet_off[tile], te = tet_off[tile + 1];
  const int vb = vtx_off[tile];
  const int nvu = vtx_off[tile + 1] - vb;
  for (int i = threadIdx.x; i < nvu; i += kTileTets) {
    const int v = vtx[vb + i];
    sid[i] = v;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      su[c][i] = io.u[(size_t)c * nv + v];
      if (KV) {
        sw[c][i] = io.w[(size_t)c * nv + v];
        sk[c][i] = T(0);
      }
      if (FO) sf[c][i] = T(0);
      if (DG) sd[c][i] = T(0);
    }
  }
  __syncthreads();
  const int t = tb + threadIdx.x;
  if (t < te) {
    const uchar4 sl4 = slots[t];
    const int sl[4] = {sl4.x, sl4.y, sl4.z, sl4.w};
    T B[9], V, mu, lam;
    load_tet(s, nt, t, mu0, lam0, B, V, mu, lam);
    T Du[9], Dw[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T u0 = su[c][sl[0]];
#pragma unroll
      for (int j = 0; j < 3; ++j) Du[c * 3 + j] = su[c][sl[j + 1]] - u0;
      if (KV) {
        const T w0 = sw[c][sl[0]];
#pragma unroll
        for (int j = 0; j < 3; ++j) Dw[c * 3 + j] = sw[c][sl[j + 1]] - w0;
      }
    }
    T fo[4][3], ko[4][3], dgo[4][3];
    if (element_eval<T, MODEL, OPS>(B, V, mu, lam, Du, Dw, fo, ko, dgo)) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (FO) atomicAdd(&sf[c][sl[a]], fo[a][c]);
          if (KV) atomicAdd(&sk[c][sl[a]], ko[a][c]);
          if (DG) atomicAdd(&sd[c][sl[a]], dgo[a][c]);
        }
      }
    } else {
      raise_error(err, EBB_ERR_INVERTED, perm[t]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nvu; i += kTileTets) {
    const int v = sid[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * nv + v;
      if (FO) atomicAdd(io.f + o, sf[c][i]);
      if (KV) atomicAdd(io.Kw + o, sk[c][i]);
      if (DG) atomicAdd(io.d + o, sd[c][i]);
    }
  }
}

template <typename T, int MODEL, int OPS, bool ATOMIC>
cudaError_t launch_range(int b, int e, int nt, int nv, const int4* keys, const int* perm, const TetStreams<T>& s,
                         T mu0, T lam0, const MapIO<T>& io, const int* active, int* err, cudaStream_t stream) {
  const int n = e - b;
  if (n <= 0) return cudaSuccess;
  const int grid = (n + kMapThreads - 1) / kMapThreads;
  tet_map_kernel<T, MODEL, OPS, ATOMIC><<<grid, kMapThreads, 0, stream>>>(b, e, nt, nv, keys, perm, s, mu0, lam0,
                                                                          io, active, err);
  return cudaGetLastError();
}

template <typename T>
const TetStreams<T>& streams_of(const ebb_rel_s* rel, bool coloured);
template <>
const TetStreams<double>& streams_of<double>(const ebb_rel_s* rel, bool coloured) {
  return coloured ? rel->colour.s64 : rel->s64;
}
template <>
const TetStreams<float>& streams_of<float>(const ebb_rel_s* rel, bool coloured) {
  return coloured ? rel->colour.s32 : rel->s32;
}

template <typename T, int MODEL, int OPS>
cudaError_t dispatch_reduce(ebb_rel_s* rel, ebb_reduce_t reduce, T mu0, T lam0, const MapIO<T>& io,
                            const int* active, cudaStream_t stream) {
  const int nt = (int)rel->size;
  const int nv = (int)rel->verts->size;
  int* err = rel->ctx->d_err;
  if (reduce == EBB_REDUCE_COLOR) {
    const Colouring& col = rel->colour;
    const TetStreams<T>& s = streams_of<T>(rel, true);
    for (int c = 0; c < col.ncolours; ++c) {
      cudaError_t e = launch_range<T, MODEL, OPS, false>(col.offsets[c], col.offsets[c + 1], nt, nv, col.keys,
                                                         col.perm, s, mu0, lam0, io, active, err, stream);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (reduce == EBB_REDUCE_TILED) {
    const Tiles& tl = rel->tiles;
    if (tl.ntiles == 0) return cudaSuccess;
    tet_tile_kernel<T, MODEL, OPS><<<tl.ntiles, kTileTets, 0, stream>>>(
        nt, nv, tl.tet_off, tl.vtx_off, tl.vtx, tl.slots, rel->tet_perm, streams_of<T>(rel, false), mu0, lam0, io,
        active, err);
    return cudaGetLastError();
  }
  return launch_range<T, MODEL, OPS, true>(0, nt, nt, nv, rel->keys, rel->tet_perm, streams_of<T>(rel, false), mu0,
                                           lam0, io, active, err, stream);
}

template <typename T, int MODEL>
cudaError_t dispatch_ops(ebb_rel_s* rel, int ops, ebb_reduce_t reduce, T mu0, T lam0, const MapIO<T>& io,
                         const int* active, cudaStream_t stream) {
  switch (ops) {
    case OP_FORCE: return dispatch_reduce<T, MODEL, OP_FORCE>(rel, reduce, mu0, lam0, io, active, stream);
    case OP_KV: return dispatch_reduce<T, MODEL, OP_KV>(rel, reduce, mu0, lam0, io, active, stream);
    case OP_FORCE | OP_KV:
      return dispatch_reduce<T, MODEL, OP_FORCE | OP_KV>(rel, reduce, mu0, lam0, io, active, stream);
    case OP_DIAG: return dispatch_reduce<T, MODEL, OP_DIAG>(rel, reduce, mu0, lam0, io, active, stream);
    case OP_FORCE | OP_KV | OP_DIAG:
      return dispatch_reduce<T, MODEL, OP_FORCE | OP_KV | OP_DIAG>(rel, reduce, mu0, lam0, io, active, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_tet_map(ebb_rel_s* rel, int model, int ops, ebb_reduce_t reduce, T mu0, T lam0,
                           const MapIO<T>& io, const int* active, cudaStream_t stream) {
  if (rel->size == 0) return cudaSuccess;
  if (model == EBB_STVK) return dispatch_ops<T, EBB_STVK>(rel, ops, reduce, mu0, lam0, io, active, stream);
  return dispatch_ops<T, EBB_NEOHOOKEAN>(rel, ops, reduce, mu0, lam0, io, active, stream);
}

template cudaError_t launch_tet_map<double>(ebb_rel_s*, int, int, ebb_reduce_t, double, double,
                                            const MapIO<double>&, const int*, cudaStream_t);
template cudaError_t launch_tet_map<float>(ebb_rel_s*, int, int, ebb_reduce_t, float, float,
                                           const MapIO<float>&, const int*, cudaStream_t);

}  // namespace ebb
