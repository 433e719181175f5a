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
//   tiled   persistent CTAs over tiles of Morton-ordered tets; each tile's
//           per-tet data arrives as one bulk copy into shared memory, its
//           distinct vertices are gathered once, per-corner results go to
//           shared memory, each distinct vertex sums its entries in a fixed
//           order (no shared-memory atomics) and gets one add per component --
//           a plain add when no other tile touches the vertex, a global atomic
//           otherwise.
#include <cstdint>

#include "async_copy.cuh"
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

// ---- tiled: persistent CTAs, one tile blob per bulk copy ---------------------
// Each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...  Two blob
// buffers alternate: while tile i is computed, the blob of tile i+G is in
// flight (cp.async.bulk on an mbarrier) and the vertex values of tile i+G are
// being loaded into registers.  Per tile:
//   phase 1  one tet per thread: corner values from the slot arrays su/sw,
//            per-corner outputs to so[NO][4][kTileTets] (conflict-free);
//   phase 2  one slot per thread: sum the slot's (corner, tet) entries in a
//            fixed order, then one atomic add per component into the vertex
//            field (a fire-and-forget reduction: no load on the critical path).
// Dynamic shared memory: blob[2] | slot values[2] (su[3][S], then sw[3][S] for
// K w) | so[NO][4][TT] | mbarrier[2].  Slot values are double buffered so the
// next tile's vertex values can be stored before the current tile's
// reduction; two barriers per tile.
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

template <typename T, int OPS>
struct TileSmem {
  static constexpr bool FO = (OPS & OP_FORCE) != 0;
  static constexpr bool KV = (OPS & OP_KV) != 0;
  static constexpr bool DG = (OPS & OP_DIAG) != 0;
  static constexpr int NO = (FO ? 3 : 0) + (KV ? 3 : 0) + (DG ? 3 : 0);
  static constexpr int S = kTileSlots;
  static constexpr int TT = kTileTets;
  static constexpr size_t slot_elems = 3 * S * (KV ? 2 : 1);  // su (+ sw) for one tile
  static constexpr size_t fixed = sizeof(T) * 2 * slot_elems + sizeof(T) * NO * 4 * TT + 2 * sizeof(uint64_t);
  static size_t bytes(const BlobLayout& L) { return 2 * (size_t)L.bytes + fixed; }
};

template <typename T, int MODEL, int OPS>
__global__ void __launch_bounds__(kTileTets)
tet_tile_kernel(int ntiles, int nv, const unsigned char* __restrict__ blobs, BlobLayout L,
                const int* __restrict__ perm, T mu0, T lam0, MapIO<T> io, const int* active, int* err) {
  using Z = TileSmem<T, OPS>;
  constexpr int S = Z::S, TT = Z::TT, NO = Z::NO;
  extern __shared__ __align__(128) unsigned char smem[];
  T* slotv = reinterpret_cast<T*>(smem + 2 * (size_t)L.bytes);
  T* so = slotv + 2 * Z::slot_elems;
  uint64_t* bar = reinterpret_cast<uint64_t*>(so + NO * 4 * TT);

  if (active != nullptr && *active == 0) return;
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  int tile = blockIdx.x;
  if (tile >= ntiles) return;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // Per-buffer state, kept in scalars (no local-memory arrays).
  bool pend0 = true, pend1 = tile + G < ntiles;
  unsigned par0 = 0u, par1 = 0u;
  if (tid == 0) {
    bulk_load(smem, blobs + (size_t)tile * L.bytes, L.bytes, &bar[0]);
    if (pend1) bulk_load(smem + L.bytes, blobs + (size_t)(tile + G) * L.bytes, L.bytes, &bar[1]);
  }
  bool bad = !mbar_wait(&bar[0], par0, kWaitCycles);
  if (__syncthreads_or(bad)) goto drain;
  pend0 = false;
  par0 ^= 1u;
  {
    const int4 h = *reinterpret_cast<const int4*>(smem);
    if (tid < h.y) {
      const int v = reinterpret_cast<const int*>(smem + kBlobVtx)[tid];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        slotv[c * S + tid] = io.u[(size_t)c * nv + v];
        if (Z::KV) slotv[(3 + c) * S + tid] = io.w[(size_t)c * nv + v];
      }
    }
  }
  __syncthreads();

  for (int k = 0;; ++k) {
    const int b = k & 1;
    const T* su = slotv + (b ? Z::slot_elems : 0);
    const T* sw = su + 3 * S;
    T* su_next = slotv + (b ? 0 : Z::slot_elems);
    unsigned char* cur = b ? smem + L.bytes : smem;
    unsigned char* nxt = b ? smem : smem + L.bytes;
    const int next = tile + G;
    // Next tile: wait for its blob, start loading its vertex values.
    T pu[3], pw[3];
    int nvu_next = 0;
    if (next < ntiles) {
      bad = !mbar_wait(&bar[b ^ 1], b ? par0 : par1, kWaitCycles);
      if (__syncthreads_or(bad)) goto drain;
      if (b) {
        pend0 = false;
        par0 ^= 1u;
      } else {
        pend1 = false;
        par1 ^= 1u;
      }
      nvu_next = reinterpret_cast<const int4*>(nxt)->y;
      if (tid < nvu_next) {
        const int v = reinterpret_cast<const int*>(nxt + kBlobVtx)[tid];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pu[c] = io.u[(size_t)c * nv + v];
          if (Z::KV) pw[c] = io.w[(size_t)c * nv + v];
        }
      }
    }
    const int4 h = *reinterpret_cast<const int4*>(cur);

    // Phase 1: one tet per thread.
    if (tid < h.x) {
      const uchar4 sl4 = reinterpret_cast<const uchar4*>(cur + kBlobSlots)[tid];
      const int sl[4] = {sl4.x, sl4.y, sl4.z, sl4.w};
      const T* Bs = reinterpret_cast<const T*>(cur + L.B);
      T B[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) B[i] = Bs[i * TT + tid];
      const T V = reinterpret_cast<const T*>(cur + L.V)[tid];
      const T mu = L.mu >= 0 ? reinterpret_cast<const T*>(cur + L.mu)[tid] : mu0;
      const T lam = L.lam >= 0 ? reinterpret_cast<const T*>(cur + L.lam)[tid] : lam0;
      T Du[9], Dw[9];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T u0 = su[c * S + sl[0]];
#pragma unroll
        for (int j = 0; j < 3; ++j) Du[c * 3 + j] = su[c * S + sl[j + 1]] - u0;
        if (Z::KV) {
          const T w0 = sw[c * S + sl[0]];
#pragma unroll
          for (int j = 0; j < 3; ++j) Dw[c * 3 + j] = sw[c * S + sl[j + 1]] - w0;
        }
      }
      T fo[4][3], ko[4][3], dgo[4][3];
      const bool ok = element_eval<T, MODEL, OPS>(B, V, mu, lam, Du, Dw, fo, ko, dgo);
      if (!ok) raise_error(err, EBB_ERR_INVERTED, perm[h.z + tid]);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          int o = 0;
          if (Z::FO) so[((o + c) * 4 + a) * TT + tid] = ok ? fo[a][c] : T(0);
          if (Z::FO) o += 3;
          if (Z::KV) so[((o + c) * 4 + a) * TT + tid] = ok ? ko[a][c] : T(0);
          if (Z::KV) o += 3;
          if (Z::DG) so[((o + c) * 4 + a) * TT + tid] = ok ? dgo[a][c] : T(0);
        }
      }
    }
    if (tid < nvu_next) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        su_next[c * S + tid] = pu[c];
        if (Z::KV) su_next[(3 + c) * S + tid] = pw[c];
      }
    }
    __syncthreads();

    // Phase 2: one distinct vertex per thread.
    if (tid < h.y) {
      const unsigned short* eoff = reinterpret_cast<const unsigned short*>(cur + kBlobEoff);
      const unsigned short* ent = reinterpret_cast<const unsigned short*>(cur + kBlobEnt);
      const int e0 = eoff[tid] & 0x7fff, e1 = eoff[tid + 1] & 0x7fff;
      T acc[NO];
#pragma unroll
      for (int o = 0; o < NO; ++o) acc[o] = T(0);
      for (int e = e0; e < e1; ++e) {
        const int code = ent[e];
        const int idx = (code >> 8) * TT + (code & 255);
#pragma unroll
        for (int o = 0; o < NO; ++o) acc[o] += so[o * 4 * TT + idx];
      }
      const int v = reinterpret_cast<const int*>(cur + kBlobVtx)[tid];
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        T* field;
        int c;
        if (Z::FO && o < 3) {
          field = io.f;
          c = o;
        } else if (Z::KV && o < (Z::FO ? 6 : 3)) {
          field = io.Kw;
          c = o - (Z::FO ? 3 : 0);
        } else {
          field = io.d;
          c = o - (Z::FO ? 3 : 0) - (Z::KV ? 3 : 0);
        }
        atomicAdd(field + (size_t)c * nv + v, acc[o]);
      }
    }
    __syncthreads();

    // The current buffer is free: refill it with the tile after next.
    if (next + G < ntiles) {
      if (tid == 0) {
        fence_proxy_async_smem();
        bulk_load(cur, blobs + (size_t)(next + G) * L.bytes, L.bytes, &bar[b]);
      }
      if (b)
        pend1 = true;
      else
        pend0 = true;
    }
    if (next >= ntiles) break;
    tile = next;
  }
  return;

drain:
  // A copy did not complete in time: report it and wait (bounded) for the
  // copies still in flight before the CTA's shared memory goes away.
  if (tid == 0) raise_error(err, EBB_ERR_TIMEOUT, blockIdx.x);
  if (pend0) mbar_wait(&bar[0], par0, kWaitCycles);
  if (pend1) mbar_wait(&bar[1], par1, kWaitCycles);
}

template <typename T, int MODEL, int OPS>
struct TileLaunchCfg {
  static size_t smem;
  static int grid_per_sm;
};
template <typename T, int MODEL, int OPS>
size_t TileLaunchCfg<T, MODEL, OPS>::smem = 0;
template <typename T, int MODEL, int OPS>
int TileLaunchCfg<T, MODEL, OPS>::grid_per_sm = 0;

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

template <typename T, int MODEL, int OPS>
cudaError_t configure_tiles() {
  cudaError_t e = cudaFuncSetAttribute(tet_tile_kernel<T, MODEL, OPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tet_tile_kernel<T, MODEL, OPS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

template <typename T, int MODEL>
cudaError_t configure_tiles_model() {
  cudaError_t e = configure_tiles<T, MODEL, OP_FORCE>();
  if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_KV>();
  if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_FORCE | OP_KV>();
  if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_DIAG>();
  if (e == cudaSuccess) e = configure_tiles<T, MODEL, OP_FORCE | OP_KV | OP_DIAG>();
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

template <typename T, int MODEL, int OPS>
cudaError_t launch_tiles(ebb_rel_s* rel, T mu0, T lam0, const MapIO<T>& io, const int* active,
                         cudaStream_t stream) {
  const Tiles& tl = rel->tiles;
  if (tl.ntiles == 0) return cudaSuccess;
  const BlobLayout& L = layout_of<T>(tl);
  const size_t smem = TileSmem<T, OPS>::bytes(L);
  using Cfg = TileLaunchCfg<T, MODEL, OPS>;
  if (Cfg::smem != smem) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tet_tile_kernel<T, MODEL, OPS>,
                                                                  kTileTets, smem);
    if (e != cudaSuccess) return e;
    Cfg::grid_per_sm = per_sm > 0 ? per_sm : 1;
    Cfg::smem = smem;
  }
  int grid = Cfg::grid_per_sm * sm_count();
  if (grid > tl.ntiles) grid = tl.ntiles;
  tet_tile_kernel<T, MODEL, OPS><<<grid, kTileTets, smem, stream>>>(tl.ntiles, (int)rel->verts->size,
                                                                    blob_of<T>(tl), L, rel->tet_perm, mu0, lam0,
                                                                    io, active, rel->ctx->d_err);
  return cudaGetLastError();
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
  if (reduce == EBB_REDUCE_TILED) return launch_tiles<T, MODEL, OPS>(rel, mu0, lam0, io, active, stream);
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
  if (rel->size == 0) return cudaSuccess;
  if (model == EBB_STVK) return dispatch_ops<T, EBB_STVK>(rel, ops, reduce, mu0, lam0, io, active, stream);
  return dispatch_ops<T, EBB_NEOHOOKEAN>(rel, ops, reduce, mu0, lam0, io, active, stream);
}

template cudaError_t launch_tet_map<double>(ebb_rel_s*, int, int, ebb_reduce_t, double, double,
                                            const MapIO<double>&, const int*, cudaStream_t);
template cudaError_t launch_tet_map<float>(ebb_rel_s*, int, int, ebb_reduce_t, float, float,
                                           const MapIO<float>&, const int*, cudaStream_t);

}  // namespace ebb
