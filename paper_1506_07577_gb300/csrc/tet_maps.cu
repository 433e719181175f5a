// Element maps over the tets relation: elastic force, K w and diag(K),
// reduced (+=) into vertex fields.
//
// A map is Ebb's kernel over a relation (Section 4.1): one instance per tet
// reads the tet's four vertex keys (tets.v[4], Section 5.2), gathers vertex
// fields through them and reduces per-corner results into vertex fields.
// Field reductions use hardware atomics (Section 6.2 "Reductions"), or, in
// the coloured variant, plain read-modify-write one colour at a time.
#include <cstdint>

#include "ebb_internal.h"
#include "tet_math.cuh"

namespace ebb {

namespace {

constexpr int kMapThreads = 128;

template <typename T, bool ATOMIC>
__device__ __forceinline__ void scatter_add(T* p, T v) {
  if (ATOMIC)
    atomicAdd(p, v);
  else
    *p += v;
}

__device__ __forceinline__ void raise_error(int* err, int code, int index) {
  if (atomicCAS(err + ERRW_CODE, 0, code) == 0) err[ERRW_INDEX] = index;
}

template <typename T, int MODEL, int OPS, bool ATOMIC>
__global__ void __launch_bounds__(kMapThreads)
tet_map_kernel(int t_begin, int t_end, int nt, int nv, const int4* __restrict__ keys,
               TetStreams<T> s, T mu0, T lam0, MapIO<T> io, const int* active, int* err) {
  if (active != nullptr && *active == 0) return;
  const int t = t_begin + blockIdx.x * kMapThreads + threadIdx.x;
  if (t >= t_end) return;

  const int4 k4 = keys[t];
  const int kk[4] = {k4.x, k4.y, k4.z, k4.w};
  T B[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i] = s.B[(size_t)i * nt + t];
  const T V = s.V[t];
  const T mu = s.mu ? s.mu[t] : mu0;
  const T lam = s.lam ? s.lam[t] : lam0;

  // G = Du B
  T G[9];
  {
    T Du[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* uc = io.u + (size_t)c * nv;
      const T u0 = uc[kk[0]];
#pragma unroll
      for (int j = 0; j < 3; ++j) Du[c * 3 + j] = uc[kk[j + 1]] - u0;
    }
    mm(Du, B, G);
  }

  StvkState<T> sv;
  NhState<T> sn;
  if (MODEL == EBB_STVK) {
    stvk_state(G, mu, lam, sv);
  } else {
    if (!nh_state(G, sn)) {
      raise_error(err, EBB_ERR_INVERTED, t);
      return;
    }
  }

  if (OPS & OP_FORCE) {
    T P[9];
    if (MODEL == EBB_STVK)
      stvk_P(sv, P);
    else
      nh_P(sn, mu, lam, P);
    // f_a = -V P b_a (b_a = row a-1 of B), f_0 = -sum
    T f0[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 1; a <= 3; ++a) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T val = -V * (P[c * 3 + 0] * B[(a - 1) * 3 + 0] + P[c * 3 + 1] * B[(a - 1) * 3 + 1] +
                            P[c * 3 + 2] * B[(a - 1) * 3 + 2]);
        f0[c] -= val;
        scatter_add<T, ATOMIC>(io.f + (size_t)c * nv + kk[a], val);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) scatter_add<T, ATOMIC>(io.f + (size_t)c * nv + kk[0], f0[c]);
  }

  if (OPS & OP_KV) {
    T dF[9];
    {
      T Dw[9];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T* wc = io.w + (size_t)c * nv;
        const T w0 = wc[kk[0]];
#pragma unroll
        for (int j = 0; j < 3; ++j) Dw[c * 3 + j] = wc[kk[j + 1]] - w0;
      }
      mm(Dw, B, dF);
    }
    T dP[9];
    if (MODEL == EBB_STVK)
      stvk_dP(sv, mu, lam, dF, dP);
    else
      nh_dP(sn, mu, lam, dF, dP);
    T k0[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 1; a <= 3; ++a) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T val = V * (dP[c * 3 + 0] * B[(a - 1) * 3 + 0] + dP[c * 3 + 1] * B[(a - 1) * 3 + 1] +
                           dP[c * 3 + 2] * B[(a - 1) * 3 + 2]);
        k0[c] -= val;
        scatter_add<T, ATOMIC>(io.Kw + (size_t)c * nv + kk[a], val);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) scatter_add<T, ATOMIC>(io.Kw + (size_t)c * nv + kk[0], k0[c]);
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
      for (int c = 0; c < 3; ++c) scatter_add<T, ATOMIC>(io.d + (size_t)c * nv + kk[a], V * dg[c]);
    }
  }
}

template <typename T, int MODEL, int OPS, bool ATOMIC>
cudaError_t launch_range(int b, int e, int nt, int nv, const int4* keys, const TetStreams<T>& s,
                         T mu0, T lam0, const MapIO<T>& io, const int* active, int* err,
                         cudaStream_t stream) {
  const int n = e - b;
  if (n <= 0) return cudaSuccess;
  const int grid = (n + kMapThreads - 1) / kMapThreads;
  tet_map_kernel<T, MODEL, OPS, ATOMIC><<<grid, kMapThreads, 0, stream>>>(b, e, nt, nv, keys, s, mu0, lam0,
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
                                                         s, mu0, lam0, io, active, err, stream);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  return launch_range<T, MODEL, OPS, true>(0, nt, nt, nv, rel->keys, streams_of<T>(rel, false), mu0, lam0, io,
                                           active, err, stream);
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
