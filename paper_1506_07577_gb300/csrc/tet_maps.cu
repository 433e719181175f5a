// Element maps over the tets relation: elastic force, K w and diag(K),
// reduced (+=) into vertex fields.
//
// A map is Ebb's kernel over a relation (Section 4.1): one instance per tet
// reads the tet's four vertex keys (tets.v[4], Section 5.2), gathers vertex
// fields through them and reduces per-corner results into vertex fields.
// The reduction strategies share one element evaluation (element.cuh):
//   direct  one thread per tet, hardware atomic adds (Section 6.2
//           "Reductions"), or plain read-modify-write inside one colour of a
//           vertex-conflict colouring (Section 7.4, Liszt's colouring);
//   tiled   persistent CTAs over tiles of Morton-ordered tets; each tile's
//           per-tet data arrives as one bulk copy into shared memory, its
//           distinct vertices are gathered once (asynchronously, by a
//           producer warp), per-corner results go to shared memory, and each
//           distinct vertex sums its entries in a fixed order (no
//           shared-memory atomics) and gets one global atomic add per
//           component (CTA machinery in tile_map.cuh);
//   tiled ordered  the tiled map with each vertex run total stored to a
//           partial row of its own instead of added atomically, then one
//           thread per vertex adds its rows in tile order (deterministic);
//   gather  per-corner outputs to a buffer, then one thread per vertex sums
//           its entries in index order (below).
#include <cstdint>

#include "async_copy.cuh"
#include "coop.cuh"
#include "ebb_internal.h"
#include "element.cuh"
#include "tet_io.cuh"
#include "tile_map.cuh"

namespace ebb {

namespace {

constexpr int kMapThreads = 128;

// ---- direct: one thread per tet -------------------------------------------
// AOS: vertex-interleaved operands (MapIO::aos, FP32): one 16-byte load per
// corner and field, one vector atomic (or one 16-byte read-modify-write)
// per corner and output.
template <typename T, int MODEL, int OPS, bool ATOMIC, bool AOS>
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
  load_edges<T, OPS, AOS>(io, nv, kk, Du, Dw);
  T fo[4][3], ko[4][3], dgo[4][3];
  if (!element_eval<T, MODEL, OPS>(B, V, mu, lam, Du, Dw, fo, ko, dgo)) {
    raise_error(err, EBB_ERR_INVERTED, perm[t]);
    return;
  }
  if constexpr (AOS) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const T* vals[3] = {fo[a], ko[a], dgo[a]};
      T* outs[3] = {io.f, io.Kw, io.d};
      const int on[3] = {OPS & OP_FORCE, OPS & OP_KV, OPS & OP_DIAG};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (!on[k]) continue;
        float* p = outs[k] + 4 * (size_t)kk[a];
        if (ATOMIC) {
          red_add_v4(p, vals[k][0], vals[k][1], vals[k][2]);
        } else {
          float4 x = *reinterpret_cast<float4*>(p);
          x.x += vals[k][0];
          x.y += vals[k][1];
          x.z += vals[k][2];
          *reinterpret_cast<float4*>(p) = x;
        }
      }
    }
  } else {
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
}

// ---- gather: per-corner outputs, then a per-vertex sum (GroupBy) ----------
// Pass 1, one thread per tet: the element's outputs go to a per-relation
// buffer instead of the vertex fields; entry 4 t + a (corner a of internal
// tet t) holds its NF output fields x 3 components, component-major with the
// fields interleaved, so that a tet's 4 entries are 12 NF contiguous values.
// Pass 2, one thread per vertex (vertices taken in the order of their first
// tet, for locality): the entries that the vertex index lists for vertex v
// (Section 6.1's GroupBy: the key-field tets.v inverted into vertex ->
// (tet, corner) rows, in increasing row order) are summed in that order and
// added into the output fields with a plain read-modify-write.
// No atomics, and every run forms the same sums in the same order: the
// result is bitwise reproducible.  An inverted element contributes zeros.
template <int OPS>
constexpr int ops_nf() {
  return ((OPS & OP_FORCE) ? 1 : 0) + ((OPS & OP_KV) ? 1 : 0) + ((OPS & OP_DIAG) ? 1 : 0);
}

template <typename T, int MODEL, int OPS, bool AOS>
__global__ void __launch_bounds__(kMapThreads)
tet_corner_kernel(int nt, int nv, const int4* __restrict__ keys, const int* __restrict__ perm, TetStreams<T> s,
                  T mu0, T lam0, MapIO<T> io, T* __restrict__ corner, const int* active, int* err) {
  constexpr int NF = ops_nf<OPS>();
  if (active != nullptr && *active == 0) return;
  const int t = blockIdx.x * kMapThreads + threadIdx.x;
  if (t >= nt) return;
  const int4 k4 = keys[t];
  const int kk[4] = {k4.x, k4.y, k4.z, k4.w};
  T B[9], V, mu, lam;
  load_tet(s, nt, t, mu0, lam0, B, V, mu, lam);
  T Du[9], Dw[9];
  load_edges<T, OPS, AOS>(io, nv, kk, Du, Dw);
  T fo[4][3], ko[4][3], dgo[4][3];
  T vals[12 * NF];
  if (element_eval<T, MODEL, OPS>(B, V, mu, lam, Du, Dw, fo, ko, dgo)) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        int f = 0;
        if (OPS & OP_FORCE) vals[(a * 3 + c) * NF + f++] = fo[a][c];
        if (OPS & OP_KV) vals[(a * 3 + c) * NF + f++] = ko[a][c];
        if (OPS & OP_DIAG) vals[(a * 3 + c) * NF + f++] = dgo[a][c];
      }
  } else {
    raise_error(err, EBB_ERR_INVERTED, perm[t]);
#pragma unroll
    for (int i = 0; i < 12 * NF; ++i) vals[i] = T(0);
  }
  // 12 NF values = 48 NF (FP32) or 96 NF (FP64) bytes: whole 16-byte stores.
  constexpr int PER16 = 16 / (int)sizeof(T);
  T* dst = corner + (size_t)t * 12 * NF;
#pragma unroll
  for (int i = 0; i < 12 * NF; i += PER16) {
    if constexpr (sizeof(T) == 4)
      *reinterpret_cast<float4*>(dst + i) = make_float4((float)vals[i], (float)vals[i + 1], (float)vals[i + 2],
                                                        (float)vals[i + 3]);
    else
      *reinterpret_cast<double2*>(dst + i) = make_double2((double)vals[i], (double)vals[i + 1]);
  }
}

constexpr int kSumThreads = 256;

template <typename T, int NF, bool AOS>
__global__ void __launch_bounds__(kSumThreads)
vertex_sum_kernel(int nv, const int* __restrict__ off, const int* __restrict__ ent, const int* __restrict__ order,
                  const T* __restrict__ corner, T* out0, T* out1, T* out2, const int* active) {
  if (active != nullptr && *active == 0) return;
  const int i = blockIdx.x * kSumThreads + threadIdx.x;
  if (i >= nv) return;
  const int v = order[i];
  T acc[3 * NF];
#pragma unroll
  for (int k = 0; k < 3 * NF; ++k) acc[k] = T(0);
  const int e0 = off[v], e1 = off[v + 1];
#pragma unroll 4
  for (int e = e0; e < e1; ++e) {
    const T* p = corner + (size_t)__ldg(ent + e) * 3 * NF;
    if constexpr (NF == 2 && sizeof(T) == 4) {
      // (f, K w) pairs: one 8-byte load per component
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 q = __ldg(reinterpret_cast<const float2*>(p) + c);
        acc[2 * c] += (T)q.x;
        acc[2 * c + 1] += (T)q.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 3 * NF; ++k) acc[k] += __ldg(p + k);
    }
  }
  T* outs[3] = {out0, out1, out2};
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    if constexpr (AOS) {
      float4* o = reinterpret_cast<float4*>(outs[f]) + v;
      float4 x = *o;
      x.x += (float)acc[f];
      x.y += (float)acc[NF + f];
      x.z += (float)acc[2 * NF + f];
      *o = x;
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) outs[f][(size_t)c * nv + v] += acc[c * NF + f];
    }
  }
}

// Second pass of the ordered tiled variant: vertex vtx[i] adds its partial
// rows off[i] .. off[i+1] (NF groups of x, y, z, 0; consecutive, in tile
// order) into the fields.
template <typename T, int NF, bool AOS>
__global__ void __launch_bounds__(kSumThreads)
partial_sum_kernel(int n, int nv, const int* __restrict__ off, const int* __restrict__ vtx,
                   const T* __restrict__ part, T* out0, T* out1, T* out2, const int* active) {
  if (active != nullptr && *active == 0) return;
  const int i = blockIdx.x * kSumThreads + threadIdx.x;
  if (i >= n) return;
  const int v = vtx[i];
  T acc[NF][3];
#pragma unroll
  for (int f = 0; f < NF; ++f) acc[f][0] = acc[f][1] = acc[f][2] = T(0);
  const int e0 = off[i], e1 = off[i + 1];
#pragma unroll 2
  for (int e = e0; e < e1; ++e) {
    const T* p = part + (size_t)e * (4 * NF);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if constexpr (sizeof(T) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p) + f);
        acc[f][0] += q.x;
        acc[f][1] += q.y;
        acc[f][2] += q.z;
      } else {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p + 4 * f));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p + 4 * f) + 1);
        acc[f][0] += a.x;
        acc[f][1] += a.y;
        acc[f][2] += b.x;
      }
    }
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    T* out = f == 0 ? out0 : (f == 1 ? out1 : out2);
    if constexpr (AOS) {
      float4* o = reinterpret_cast<float4*>(out) + v;
      float4 x = *o;
      x.x += (float)acc[f][0];
      x.y += (float)acc[f][1];
      x.z += (float)acc[f][2];
      *o = x;
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) out[(size_t)c * nv + v] += acc[f][c];
    }
  }
}

// ---- tiled (machinery in tile_map.cuh) ------------------------------------
// The standalone map: one pass over fresh rings.
template <typename T, int MODEL, int OPS, bool AOS, bool ORD>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 4 : 2)
tet_tile_kernel(int ntiles, int nv, const unsigned char* __restrict__ blobs, BlobLayout L,
                const int* __restrict__ perm, T mu0, T lam0, MapIO<T> io, const int* active, int* err,
                int drop_tile, long long wait_cycles) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (active != nullptr && *active == 0) return;
  const int G = gridDim.x;
  if ((int)blockIdx.x >= ntiles) return;
  const int n_my = (ntiles - (int)blockIdx.x + G - 1) / G;
  const TileView<T, OPS> V = tile_view<T, OPS>(smem, L);
  tile_init(V);
  __syncthreads();
  tile_map_pass<T, MODEL, OPS, AOS, ORD>(V, n_my, 0, nv, blobs, L, perm, mu0, lam0, io, err, drop_tile, wait_cycles);
}


template <typename T, int MODEL, int OPS, bool AOS, bool ORD>
struct TileLaunchCfg {
  static size_t smem;
  static int grid_per_sm;
};
template <typename T, int MODEL, int OPS, bool AOS, bool ORD>
size_t TileLaunchCfg<T, MODEL, OPS, AOS, ORD>::smem = 0;
template <typename T, int MODEL, int OPS, bool AOS, bool ORD>
int TileLaunchCfg<T, MODEL, OPS, AOS, ORD>::grid_per_sm = 0;

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <typename T, int MODEL, int OPS, bool AOS, bool ORD>
cudaError_t configure_tiles_one() {
  cudaError_t e = cudaFuncSetAttribute(tet_tile_kernel<T, MODEL, OPS, AOS, ORD>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tet_tile_kernel<T, MODEL, OPS, AOS, ORD>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}
template <typename T, int MODEL, int OPS, bool AOS = false>
cudaError_t configure_tiles() {
  cudaError_t e = configure_tiles_one<T, MODEL, OPS, AOS, false>();
  if (e == cudaSuccess) e = configure_tiles_one<T, MODEL, OPS, AOS, true>();
  return e;
}

template <typename T, int MODEL>
cudaError_t configure_tiles_model() {
  cudaError_t e = configure_tiles<T, MODEL, OP_FORCE>();
  if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_KV>();
  if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_FORCE | OP_KV>();
  if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_DIAG>();
  if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_FORCE | OP_KV | OP_DIAG>();
  // Vertex-interleaved variants (FP32 only).
  if constexpr (sizeof(T) == 4) {
    if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_FORCE, true>();
    if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_KV, true>();
    if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_FORCE | OP_KV, true>();
    if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_DIAG, true>();
    if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_FORCE | OP_KV | OP_DIAG, true>();
  }
  return e;
}

template <typename T>
const unsigned char* blob_of(const Tiles& tl);
template <>
const unsigned char* blob_of<float>(const Tiles& tl) { return tl.blob32; }
template <>
const unsigned char* blob_of<double>(const Tiles& tl) { return tl.blob64; }
template <typename T>
const BlobLayout& layout_of(const Tiles& tl);
template <>
const BlobLayout& layout_of<float>(const Tiles& tl) { return tl.L32; }
template <>
const BlobLayout& layout_of<double>(const Tiles& tl) { return tl.L64; }

template <typename T, int MODEL, int OPS, bool AOS, bool ORD = false>
cudaError_t launch_tiles(ebb_rel_s* rel, T mu0, T lam0, const MapIO<T>& io, const int* active,
                         cudaStream_t stream) {
  const Tiles& tl = rel->tiles;
  if (tl.ntiles == 0) return cudaSuccess;
  // A tile range is the tiles of a shorter blob array: the kernel indexes
  // tiles relative to the pointer it gets (the ordered variant's partial
  // rows are numbered from tile 0, so it always maps every tile).
  const int t0 = io.tile_begin;
  const int t1 = io.tile_end < 0 ? tl.ntiles : io.tile_end;
  if (t0 < 0 || t1 > tl.ntiles || t0 > t1 || (ORD && (t0 != 0 || t1 != tl.ntiles))) return cudaErrorInvalidValue;
  const int count = t1 - t0;
  if (count == 0) return cudaSuccess;
  const BlobLayout& L = layout_of<T>(tl);
  const size_t smem = TileSmem<T, OPS>::bytes(L);
  using Cfg = TileLaunchCfg<T, MODEL, OPS, AOS, ORD>;
  if (Cfg::smem != smem) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tet_tile_kernel<T, MODEL, OPS, AOS, ORD>,
                                                                  kTileThreads, smem);
    if (e != cudaSuccess) return e;
    Cfg::grid_per_sm = per_sm > 0 ? per_sm : 1;
    Cfg::smem = smem;
  }
  int grid = Cfg::grid_per_sm * sm_count();
  if (grid > count) grid = count;
  const int drop = rel->test_drop_tile;
  tet_tile_kernel<T, MODEL, OPS, AOS, ORD><<<grid, kTileThreads, smem, stream>>>(
      count, (int)rel->verts->size, blob_of<T>(tl) + (size_t)t0 * L.bytes, L, rel->tet_perm, mu0, lam0, io, active,
      rel->ctx->d_err, drop, drop >= 0 ? kTestWaitCycles : kWaitCycles);
  return cudaGetLastError();
}

// Partial rows of the ordered tiled variant (room for three outputs),
// allocated at first use and kept with the tiles; like the gather buffer,
// never allocated inside a stream capture.
template <typename T>
cudaError_t partial_buffer(ebb_rel_s* rel, cudaStream_t stream, T** out) {
  void*& buf = rel->tiles.partial[sizeof(T) == 4 ? 0 : 1];
  if (buf == nullptr) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
    e = cudaMalloc(&buf, (size_t)rel->tiles.ntiles * kTileTets * 12 * sizeof(T));
    if (e != cudaSuccess) {
      buf = nullptr;
      return e;
    }
  }
  *out = static_cast<T*>(buf);
  return cudaSuccess;
}

// The ordered tiled variant: the tiled map stores each run total to its
// partial row, then one thread per vertex adds its rows in tile order.  No
// floating-point atomics, so results repeat bit for bit.
template <typename T, int MODEL, int OPS, bool AOS>
cudaError_t launch_tiles_ordered(ebb_rel_s* rel, T mu0, T lam0, const MapIO<T>& io, const int* active,
                                 cudaStream_t stream) {
  constexpr int NF = ops_nf<OPS>();
  const Tiles& tl = rel->tiles;
  const int nv = (int)rel->verts->size;
  if (tl.ntiles == 0 || nv == 0) return cudaSuccess;
  MapIO<T> pio = io;
  pio.unit_row = tl.unit_row;
  cudaError_t e = partial_buffer<T>(rel, stream, &pio.part);
  if (e != cudaSuccess) return e;
  e = launch_tiles<T, MODEL, OPS, AOS, true>(rel, mu0, lam0, pio, active, stream);
  if (e != cudaSuccess) return e;
  T* outs[3] = {nullptr, nullptr, nullptr};
  int f = 0;
  if (OPS & OP_FORCE) outs[f++] = io.f;
  if (OPS & OP_KV) outs[f++] = io.Kw;
  if (OPS & OP_DIAG) outs[f++] = io.d;
  if (tl.n_ord == 0) return cudaSuccess;
  partial_sum_kernel<T, NF, AOS><<<(tl.n_ord + kSumThreads - 1) / kSumThreads, kSumThreads, 0, stream>>>(
      tl.n_ord, nv, tl.ord_off, tl.ord_vtx, pio.part, outs[0], outs[1], outs[2], active);
  return cudaGetLastError();
}

template <typename T, int MODEL, int OPS, bool ATOMIC>
cudaError_t launch_range(int b, int e, int nt, int nv, const int4* keys, const int* perm, const TetStreams<T>& s,
                         T mu0, T lam0, const MapIO<T>& io, const int* active, int* err, cudaStream_t stream) {
  const int n = e - b;
  if (n <= 0) return cudaSuccess;
  const int grid = (n + kMapThreads - 1) / kMapThreads;
  if (io.aos) {
    if constexpr (sizeof(T) == 4) {
      tet_map_kernel<T, MODEL, OPS, ATOMIC, true><<<grid, kMapThreads, 0, stream>>>(b, e, nt, nv, keys, perm, s, mu0,
                                                                                    lam0, io, active, err);
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }
  tet_map_kernel<T, MODEL, OPS, ATOMIC, false><<<grid, kMapThreads, 0, stream>>>(b, e, nt, nv, keys, perm, s, mu0,
                                                                                 lam0, io, active, err);
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

// Per-corner buffer of the gather variant: 12 x 3 values per tet (room for
// all three outputs), allocated at first use and kept with the relation.
// Never allocated inside a stream capture: the implicit steps' first map
// (force, K v and diag together) runs before their capture.
template <typename T>
cudaError_t gather_buffer(ebb_rel_s* rel, cudaStream_t stream, T** out) {
  void*& buf = rel->gather_corner[sizeof(T) == 4 ? 0 : 1];
  if (buf == nullptr) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
    e = cudaMalloc(&buf, (size_t)rel->size * 36 * sizeof(T));
    if (e != cudaSuccess) {
      buf = nullptr;
      return e;
    }
  }
  *out = static_cast<T*>(buf);
  return cudaSuccess;
}

template <typename T, int MODEL, int OPS, bool AOS>
cudaError_t launch_gather(ebb_rel_s* rel, T mu0, T lam0, const MapIO<T>& io, const int* active, cudaStream_t stream) {
  constexpr int NF = ops_nf<OPS>();
  const int nt = (int)rel->size, nv = (int)rel->verts->size;
  T* corner = nullptr;
  cudaError_t e = gather_buffer<T>(rel, stream, &corner);
  if (e != cudaSuccess) return e;
  tet_corner_kernel<T, MODEL, OPS, AOS><<<(nt + kMapThreads - 1) / kMapThreads, kMapThreads, 0, stream>>>(
      nt, nv, rel->keys, rel->tet_perm, streams_of<T>(rel, false), mu0, lam0, io, corner, active, rel->ctx->d_err);
  e = cudaGetLastError();
  if (e != cudaSuccess || nv == 0) return e;
  T* outs[3] = {nullptr, nullptr, nullptr};
  int f = 0;
  if (OPS & OP_FORCE) outs[f++] = io.f;
  if (OPS & OP_KV) outs[f++] = io.Kw;
  if (OPS & OP_DIAG) outs[f++] = io.d;
  vertex_sum_kernel<T, NF, AOS><<<(nv + kSumThreads - 1) / kSumThreads, kSumThreads, 0, stream>>>(
      nv, rel->vindex.off, rel->vindex.ent, rel->vindex.order, corner, outs[0], outs[1], outs[2], active);
  return cudaGetLastError();
}

// The cooperative variant: three lanes per tet (coop.cuh), atomic scatter.
template <typename T, int MODEL, int OPS>
cudaError_t launch_coop(ebb_rel_s* rel, T mu0, T lam0, const MapIO<T>& io, const int* active, cudaStream_t stream) {
  const int nt = (int)rel->size, nv = (int)rel->verts->size;
  const int grid = (nt + kCoopTetsPerBlock - 1) / kCoopTetsPerBlock;
  if (io.aos) {
    if constexpr (sizeof(T) == 4) {
      tet_coop_kernel<T, MODEL, OPS, true><<<grid, kCoopThreads, 0, stream>>>(
          nt, nv, rel->keys, rel->tet_perm, streams_of<T>(rel, false), mu0, lam0, io, active, rel->ctx->d_err);
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }
  tet_coop_kernel<T, MODEL, OPS, false><<<grid, kCoopThreads, 0, stream>>>(
      nt, nv, rel->keys, rel->tet_perm, streams_of<T>(rel, false), mu0, lam0, io, active, rel->ctx->d_err);
  return cudaGetLastError();
}

template <typename T, int MODEL, int OPS>
cudaError_t dispatch_reduce(ebb_rel_s* rel, ebb_reduce_t reduce, T mu0, T lam0, const MapIO<T>& io,
                            const int* active, cudaStream_t stream) {
  const int nt = (int)rel->size;
  const int nv = (int)rel->verts->size;
  int* err = rel->ctx->d_err;
  if (reduce == EBB_REDUCE_COOP) return launch_coop<T, MODEL, OPS>(rel, mu0, lam0, io, active, stream);
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
  if (reduce == EBB_REDUCE_GATHER) {
    if (io.aos) {
      if constexpr (sizeof(T) == 4) return launch_gather<T, MODEL, OPS, true>(rel, mu0, lam0, io, active, stream);
      return cudaErrorInvalidValue;
    }
    return launch_gather<T, MODEL, OPS, false>(rel, mu0, lam0, io, active, stream);
  }
  if (reduce == EBB_REDUCE_TILED) {
    if (io.aos) {
      // vertex-interleaved operands: FP32 only
      if constexpr (sizeof(T) == 4) return launch_tiles<T, MODEL, OPS, true>(rel, mu0, lam0, io, active, stream);
      return cudaErrorInvalidValue;
    }
    return launch_tiles<T, MODEL, OPS, false>(rel, mu0, lam0, io, active, stream);
  }
  if (reduce == EBB_REDUCE_TILED_ORDERED) {
    if (io.aos) {
      if constexpr (sizeof(T) == 4)
        return launch_tiles_ordered<T, MODEL, OPS, true>(rel, mu0, lam0, io, active, stream);
      return cudaErrorInvalidValue;
    }
    return launch_tiles_ordered<T, MODEL, OPS, false>(rel, mu0, lam0, io, active, stream);
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

// Opt the tiled kernels into their dynamic shared-memory sizes on the current
// device (done at finalize, never inside a stream capture).
cudaError_t prepare_map_kernels() {
  cudaError_t e = configure_tiles_model<float, EBB_STVK>();
  if (e == cudaSuccess) e = configure_tiles_model<float, EBB_NEOHOOKEAN>();
  if (e == cudaSuccess) e = configure_tiles_model<double, EBB_STVK>();
  if (e == cudaSuccess) e = configure_tiles_model<double, EBB_NEOHOOKEAN>();
  return e;
}

template <typename T>
cudaError_t launch_tet_map(ebb_rel_s* rel, int model, int ops, ebb_reduce_t reduce, T mu0, T lam0,
                           const MapIO<T>& io, const int* active, cudaStream_t stream) {
  // The assembled-stiffness operations share the maps' field handling.
  if (ops == OP_ASSEMBLE) return launch_assemble<T>(rel, model, mu0, lam0, io, stream);
  if (ops == OP_SPMV) return launch_spmv<T>(rel, io.u, io.Kw, io.aos, active, stream);
  if (rel->size == 0) return cudaSuccess;
  if (model == EBB_STVK) return dispatch_ops<T, EBB_STVK>(rel, ops, reduce, mu0, lam0, io, active, stream);
  return dispatch_ops<T, EBB_NEOHOOKEAN>(rel, ops, reduce, mu0, lam0, io, active, stream);
}

template cudaError_t launch_tet_map<double>(ebb_rel_s*, int, int, ebb_reduce_t, double, double,
                                            const MapIO<double>&, const int*, cudaStream_t);
template cudaError_t launch_tet_map<float>(ebb_rel_s*, int, int, ebb_reduce_t, float, float,
                                           const MapIO<float>&, const int*, cudaStream_t);

}  // namespace ebb
