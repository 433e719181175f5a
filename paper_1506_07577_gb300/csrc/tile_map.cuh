// The tiled map's CTA machinery (device code): shared-memory rings of tile
// blobs and gathered vertex values, the producer warp and the consumer
// phases, as one pass over a CTA's tiles (a kernel may run several passes
// over the same rings).
#pragma once

#include <cstdint>

#include "async_copy.cuh"
#include "ebb_internal.h"
#include "element.cuh"
#include "tet_io.cuh"

namespace ebb {

// ---- tiled: warp-specialised persistent CTAs over tile blobs --------------
// A CTA is kTileTets consumer threads (one tet each) plus one producer warp,
// and walks tiles blockIdx.x, blockIdx.x + G, ... (G = gridDim.x).  The
// producer keeps the consumers fed through two shared-memory rings guarded by
// mbarriers (every wait bounded):
//   blob ring  (RB stages)  each tile's whole blob -- integer prefix and
//              per-tet Dm^-1, V, Lame planes -- as one cp.async.bulk;
//   slot ring  (RV stages)  the tile's distinct vertex values (u, and w for
//              K w), gathered by the producer's 32 lanes with element-wise
//              cp.async as soon as the tile's vertex ids have landed, its
//              completion tracked by an mbarrier (LAG tiles behind the
//              blob copies).
// The consumers, per tile, with one named barrier among themselves:
//   phase 1  one tet per thread: corner values from the slot vectors, per-tet
//            floats from the blob, element evaluation, per-corner outputs to
//            shared memory (fields interleaved, conflict-free);
//                                 -- the consumers' barrier --
//            (the tile's slot vectors are released to the producer)
//   phase 2  one reduction unit per thread: the sum of at most kUnitEntries
//            entries of one vertex, in a fixed order; the units of one vertex
//            on consecutive lanes are combined by a segmented shuffle tree and
//            the run's first lane issues one atomic add per component (a
//            fire-and-forget reduction); then each warp releases the blob.
// With two per-corner output buffers phase 2 of one tile overlaps phase 1 of
// the next; with one, a second consumer barrier precedes the output stores.  Dynamic shared memory: blob ring | slot ring (u[S][4]
// then w[S][4] per stage) | outputs[2][4*3][TT+1][NF] | barriers, abort flag.
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz
constexpr long long kTestWaitCycles = 2000000LL;  // about 1 ms: waits under EBB_MAP_TEST_DROP_TILE
constexpr int kTileThreads = kTileTets + 32;

template <typename T, int OPS>
struct TileSmem {
  // Ring depths (measured): FP32 runs three blob stages and one output
  // buffer so that four CTAs fit an SM; FP64 blobs take two stages and two
  // output buffers at two CTAs per SM.
  static constexpr int RB = sizeof(T) == 4 ? 3 : 2;   // blob stages
  static constexpr int RV = 2;                        // slot-vector stages
  static constexpr int LAG = 1;                       // gathers trail blob copies by LAG tiles
  static constexpr int OB = sizeof(T) == 4 ? 1 : 2;   // per-corner output buffers
  static_assert(LAG < RB, "the producer must not wait for a blob it has not issued");
  static constexpr bool FO = (OPS & OP_FORCE) != 0;
  static constexpr bool KV = (OPS & OP_KV) != 0;
  static constexpr bool DG = (OPS & OP_DIAG) != 0;
  static constexpr int NF = (FO ? 1 : 0) + (KV ? 1 : 0) + (DG ? 1 : 0);  // output fields
  static constexpr int S = kTileSlots;
  static constexpr int TT = kTileTets;
  static constexpr size_t slot_elems = (size_t)S * 4 * (KV ? 2 : 1);
  static constexpr size_t out_elems = (size_t)4 * 3 * (TT + 1) * NF;  // rows of TT+1: column TT pads
  static constexpr int nbar = 2 * RB + 2 * RV;
  __host__ __device__ static size_t slot_off(const BlobLayout& L) { return (size_t)RB * L.bytes; }
  __host__ __device__ static size_t out_off(const BlobLayout& L) { return slot_off(L) + sizeof(T) * RV * slot_elems; }
  __host__ __device__ static size_t bar_off(const BlobLayout& L) { return out_off(L) + sizeof(T) * OB * out_elems; }
  __host__ __device__ static size_t bytes(const BlobLayout& L) { return bar_off(L) + sizeof(uint64_t) * nbar + 16; }
};

// 3-vectors stored 4 wide in shared memory.
__device__ __forceinline__ void ld3(const float* p, float* v) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
}
__device__ __forceinline__ void ld3(const double* p, double* v) {
  const double2 q = *reinterpret_cast<const double2*>(p);
  v[0] = q.x;
  v[1] = q.y;
  v[2] = p[2];
}

// NF interleaved output values at p.
template <typename T, int NF>
__device__ __forceinline__ void st_out(T* p, const T* v) {
  if (NF == 2) {
    if (sizeof(T) == 4)
      *reinterpret_cast<float2*>(p) = make_float2((float)v[0], (float)v[1]);
    else
      *reinterpret_cast<double2*>(p) = make_double2((double)v[0], (double)v[1]);
  } else {
#pragma unroll
    for (int i = 0; i < NF; ++i) p[i] = v[i];
  }
}
template <typename T, int NF>
__device__ __forceinline__ void add_out(const T* p, T* acc) {
  if (NF == 2) {
    if (sizeof(T) == 4) {
      const float2 q = *reinterpret_cast<const float2*>(p);
      acc[0] += (T)q.x;
      acc[1] += (T)q.y;
    } else {
      const double2 q = *reinterpret_cast<const double2*>(p);
      acc[0] += (T)q.x;
      acc[1] += (T)q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NF; ++i) acc[i] += p[i];
  }
}

// Shared-memory view of one CTA's tile machinery (layout of TileSmem).
template <typename T, int OPS>
struct TileView {
  unsigned char* ring;
  T* slots;
  T* outs;
  uint64_t* full_b;
  uint64_t* empty_b;
  uint64_t* full_v;
  uint64_t* empty_v;
  volatile int* abort_flag;
};

template <typename T, int OPS>
__device__ __forceinline__ TileView<T, OPS> tile_view(unsigned char* smem, const BlobLayout& L) {
  using Z = TileSmem<T, OPS>;
  TileView<T, OPS> v;
  v.ring = smem;
  v.slots = reinterpret_cast<T*>(smem + Z::slot_off(L));
  v.outs = reinterpret_cast<T*>(smem + Z::out_off(L));
  v.full_b = reinterpret_cast<uint64_t*>(smem + Z::bar_off(L));
  v.empty_b = v.full_b + Z::RB;
  v.full_v = v.empty_b + Z::RB;
  v.empty_v = v.full_v + Z::RV;
  v.abort_flag = reinterpret_cast<volatile int*>(v.empty_v + Z::RV);
  return v;
}

// Barrier initialisation by thread 0 (the caller then syncs the CTA).
template <typename T, int OPS>
__device__ __forceinline__ void tile_init(const TileView<T, OPS>& V) {
  using Z = TileSmem<T, OPS>;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int r = 0; r < Z::RB; ++r) {
      mbar_init(&V.full_b[r], 1);
      mbar_init(&V.empty_b[r], Z::TT / 32);
    }
#pragma unroll
    for (int r = 0; r < Z::RV; ++r) {
      mbar_init(&V.full_v[r], 32);
      mbar_init(&V.empty_v[r], 1);
    }
    *V.abort_flag = 0;
    fence_mbar_init();
  }
}

// One pass of the map over this CTA's tiles blockIdx.x, blockIdx.x + G, ...
// (n_my of them).  `jbase` counts the tiles this CTA went through in earlier
// passes over the same rings, so that ring stages and barrier phases carry
// on from one pass to the next.  Returns false in a thread that gave up waiting or saw the
// abort flag (the timeout is raised in `err`; the producer has drained its
// copies).  AOS: vertex-interleaved operands (MapIO::aos): the producer
// copies each vertex's 16 bytes with one cp.async, the reduction adds each
// vertex's three components with one vector atomic.  ORD: the ordered
// variant, each run total stored to its partial row (MapIO::part, row index
// MapIO::unit_row, read at the start of the tile) instead of added into the
// fields.

__device__ __forceinline__ void st_part4(float* p, float x, float y, float z) {
  *reinterpret_cast<float4*>(p) = make_float4(x, y, z, 0.f);
}
__device__ __forceinline__ void st_part4(double* p, double x, double y, double z) {
  reinterpret_cast<double2*>(p)[0] = make_double2(x, y);
  reinterpret_cast<double2*>(p)[1] = make_double2(z, 0.0);
}

template <typename T, int MODEL, int OPS, bool AOS, bool ORD>
__device__ __forceinline__ bool tile_map_pass(const TileView<T, OPS>& V, int n_my, int jbase, int nv,
                                              const unsigned char* __restrict__ blobs, const BlobLayout& L,
                                              const int* __restrict__ perm, T mu0, T lam0, const MapIO<T>& io,
                                              int* err, int drop_tile, long long wait_cycles) {
  using Z = TileSmem<T, OPS>;
  constexpr int TT = Z::TT, NF = Z::NF, RB = Z::RB, RV = Z::RV;
  unsigned char* ring = V.ring;
  T* slots = V.slots;
  T* outs = V.outs;
  uint64_t* full_b = V.full_b;
  uint64_t* empty_b = V.empty_b;
  uint64_t* full_v = V.full_v;
  uint64_t* empty_v = V.empty_v;
  volatile int* abort_flag = V.abort_flag;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int G = gridDim.x;

  if (tid >= TT) {
    // ---------------------------------------------------------- producer --
    unsigned pend = 0u, pend_parity = 0u;  // blob stages with an unwaited copy
    bool bad = false;
    for (int j = 0; j < n_my + Z::LAG && !bad; ++j) {
      if (j < n_my) {
        const int J = jbase + j;
        const int sb = J % RB;
        bool ok = J < RB || mbar_wait_or_abort(&empty_b[sb], ((J / RB) - 1) & 1u, abort_flag, wait_cycles);
        if (__any_sync(0xffffffffu, !ok)) {
          bad = true;
          break;
        }
        const int tj = (int)blockIdx.x + j * G;
        if (tj != drop_tile) {  // drop_tile: failure-detection tests only (-1 otherwise)
          if (lane == 0) {
            // Blobs are read once per map: evict them first, so that the
            // vertex fields and the CG vectors stay in L2.
            fence_proxy_async_smem();
            bulk_load_hint(ring + (size_t)sb * L.bytes, blobs + (size_t)tj * L.bytes, L.copy, &full_b[sb],
                           make_policy_evict_first());
          }
          pend |= 1u << sb;
          pend_parity = (pend_parity & ~(1u << sb)) | (((unsigned)(J / RB) & 1u) << sb);
        }
      }
      const int jj = j - Z::LAG;
      if (jj >= 0 && jj < n_my) {
        const int JJ = jbase + jj;
        const int sb = JJ % RB, sv = JJ % RV;
        bool ok = mbar_wait_or_abort(&full_b[sb], (JJ / RB) & 1u, abort_flag, wait_cycles);
        if (ok) pend &= ~(1u << sb);
        ok = ok && (JJ < RV || mbar_wait_or_abort(&empty_v[sv], ((JJ / RV) - 1) & 1u, abort_flag, wait_cycles));
        if (__any_sync(0xffffffffu, !ok)) {
          bad = true;
          break;
        }
        const unsigned char* st = ring + (size_t)sb * L.bytes;
        const int nvu = reinterpret_cast<const int4*>(st)->y;
        const int* vid = reinterpret_cast<const int*>(st + kBlobVtx);
        T* su = slots + (size_t)sv * Z::slot_elems;
        if (AOS) {
          for (int sl = lane; sl < nvu; sl += 32) {
            const int v = vid[sl];
            cp_async_16(su + 4 * sl, io.u + 4 * (size_t)v);
            if (Z::KV) cp_async_16(su + 4 * (Z::S + sl), io.w + 4 * (size_t)v);
          }
        } else {
          // Lane l copies word l + 32k of the 4-wide slot vectors (component
          // 3 is padding): consecutive lanes write consecutive shared words.
          for (int wd = lane; wd < 4 * nvu; wd += 32) {
            const int c = wd & 3;
            if (c < 3) {
              const int v = vid[wd >> 2];
              cp_async_elem(su + wd, io.u + (size_t)c * nv + v);
              if (Z::KV) cp_async_elem(su + 4 * Z::S + wd, io.w + (size_t)c * nv + v);
            }
          }
        }
        cp_async_arrive_noinc(&full_v[sv]);
      }
    }
    cp_async_wait_all();
    if (bad) {
      if (lane == 0) {
        raise_error(err, EBB_ERR_TIMEOUT, blockIdx.x);
        *abort_flag = 1;
      }
      // Bounded drain of the bulk copies still in flight before the CTA's
      // shared memory goes away.
#pragma unroll
      for (int r = 0; r < RB; ++r)
        if ((pend >> r) & 1u) mbar_wait(&full_b[r], (pend_parity >> r) & 1u, wait_cycles);
    }
    return !bad;
  }

  // ------------------------------------------------------------ consumers --
  T* out_field[3];
  {
    int f = 0;
    if (Z::FO) out_field[f++] = io.f;
    if (Z::KV) out_field[f++] = io.Kw;
    if (Z::DG) out_field[f++] = io.d;
  }
  for (int j = 0; j < n_my; ++j) {
    const int J = jbase + j;
    const int sb = J % RB, sv = J % RV;
    const unsigned char* st = ring + (size_t)sb * L.bytes;
    const T* su = slots + (size_t)sv * Z::slot_elems;
    const T* sw = su + 4 * Z::S;
    // ordered variant: this unit's partial row, loaded now and used after
    // phase 1 (the tile index is absolute: the ordered map maps every tile)
    int urow = -1;
    if constexpr (ORD) urow = __ldg(io.unit_row + ((size_t)blockIdx.x + (size_t)j * G) * TT + tid);
    T* sob = outs + (Z::OB == 2 ? (J & 1) : 0) * Z::out_elems;
    const bool ok = mbar_wait_or_abort(&full_b[sb], (J / RB) & 1u, abort_flag, wait_cycles) &&
                    mbar_wait_or_abort(&full_v[sv], (J / RV) & 1u, abort_flag, wait_cycles);
    // Phase 1: one tet per thread (skipped by a thread whose wait gave up).
    const int4 h = ok ? *reinterpret_cast<const int4*>(st) : make_int4(0, 0, 0, 0);
    T fo[4][3], ko[4][3], dgo[4][3];
    bool good = true;
    if (tid < h.x) {
      const uchar4 sl4 = reinterpret_cast<const uchar4*>(st + kBlobSlots)[tid];
      const int sl[4] = {sl4.x, sl4.y, sl4.z, sl4.w};
      T Du[9], Dw[9];
      {
        T x0[3], xa[3];
        ld3(su + 4 * sl[0], x0);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          ld3(su + 4 * sl[q + 1], xa);
#pragma unroll
          for (int c = 0; c < 3; ++c) Du[c * 3 + q] = xa[c] - x0[c];
        }
        if (Z::KV) {
          ld3(sw + 4 * sl[0], x0);
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            ld3(sw + 4 * sl[q + 1], xa);
#pragma unroll
            for (int c = 0; c < 3; ++c) Dw[c * 3 + q] = xa[c] - x0[c];
          }
        }
      }
      // The tet's Dm^-1, V, mu, lambda: from its row record in three (FP32)
      // or six (FP64) 16-byte loads, or from the field planes.
      T rec[12];
      if (L.planes) {
        // per-field planes: one coalesced load per field
        const T* R = reinterpret_cast<const T*>(st + L.rec) + tid;
#pragma unroll
        for (int k = 0; k < 10; ++k) rec[k] = R[k * TT];
        rec[10] = L.material ? R[10 * TT] : T(0);
        rec[11] = L.material ? R[11 * TT] : T(0);
      } else if constexpr (sizeof(T) == 4) {
        const float4* R = reinterpret_cast<const float4*>(st + L.rec) + 3 * tid;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float4 q = R[k];
          rec[4 * k] = q.x;
          rec[4 * k + 1] = q.y;
          rec[4 * k + 2] = q.z;
          rec[4 * k + 3] = q.w;
        }
      } else {
        const double2* R = reinterpret_cast<const double2*>(st + L.rec) + (rec_len<T>() / 2) * tid;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const double2 q = R[k];
          rec[2 * k] = q.x;
          rec[2 * k + 1] = q.y;
        }
      }
      T Bm[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) Bm[i] = rec[i];
      const T V = rec[9];
      const T mu = L.material ? rec[10] : mu0;
      const T lam = L.material ? rec[11] : lam0;
      good = element_eval<T, MODEL, OPS>(Bm, V, mu, lam, Du, Dw, fo, ko, dgo);
      if (!good) raise_error(err, EBB_ERR_INVERTED, perm[h.z + tid]);
    }
    // With one output buffer, the previous tile's phase 2 must be done with it.
    if (Z::OB == 1) named_sync_or<TT>(false);
    if (tid < h.x) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T v[NF > 0 ? NF : 1];
          int f = 0;
          if (Z::FO) v[f++] = good ? fo[a][c] : T(0);
          if (Z::KV) v[f++] = good ? ko[a][c] : T(0);
          if (Z::DG) v[f++] = good ? dgo[a][c] : T(0);
          st_out<T, NF>(sob + ((size_t)(a * 3 + c) * (TT + 1) + tid) * NF, v);
        }
      }
    }
    if (named_sync_or<TT>(!ok)) {
      if (tid == 0) {
        raise_error(err, EBB_ERR_TIMEOUT, blockIdx.x);
        *abort_flag = 1;
      }
      return false;
    }
    if (tid == 0) mbar_arrive(&empty_v[sv]);

    // Phase 2: one reduction unit per thread: kUnitEntries independent loads.
    if constexpr (sizeof(T) == 4 && NF == 2) {
      // FP32 force and K w together: each entry's (f, K w) pair is one
      // 8-byte load and one paired add; same order of additions as below.
      const uint32_t d = reinterpret_cast<const uint32_t*>(st + kBlobUnits)[tid];
      const unsigned rem = (d >> 22) & 0xfu;
      float2 acc[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] = make_float2(0.f, 0.f);
      if (d & 1u) {
        const uint4 codes = reinterpret_cast<const uint4*>(st + kBlobEnt)[tid];
        const unsigned cw[4] = {codes.x, codes.y, codes.z, codes.w};
#pragma unroll
        for (int q = 0; q < kUnitEntries; ++q) {
          const unsigned code = (cw[q >> 1] >> (16 * (q & 1))) & 0xffffu;
          if (code != kEntryNone) {
            const float* p = reinterpret_cast<const float*>(sob) + (size_t)code * 2;
#pragma unroll
            for (int c = 0; c < 3; ++c)
              acc[c] = __fadd2_rn(acc[c], *reinterpret_cast<const float2*>(p + c * (TT + 1) * 2));
          }
        }
      }
      const unsigned maxrem = __reduce_max_sync(0xffffffffu, rem);
      for (unsigned stp = 1; stp <= maxrem; stp <<= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 x = make_float2(__shfl_down_sync(0xffffffffu, acc[c].x, stp),
                                       __shfl_down_sync(0xffffffffu, acc[c].y, stp));
          if (rem >= stp) acc[c] = __fadd2_rn(acc[c], x);
        }
      }
      if ((d >> 26) & 1u) {
        const int v = reinterpret_cast<const int*>(st + kBlobVtx)[(d >> 14) & 0xffu];
        if constexpr (ORD) {
          float* row = reinterpret_cast<float*>(io.part) + (size_t)urow * 8;
          *reinterpret_cast<float4*>(row) = make_float4(acc[0].x, acc[1].x, acc[2].x, 0.f);
          *reinterpret_cast<float4*>(row + 4) = make_float4(acc[0].y, acc[1].y, acc[2].y, 0.f);
        } else if constexpr (AOS) {
          red_add_v4(reinterpret_cast<float*>(out_field[0]) + 4 * (size_t)v, acc[0].x, acc[1].x, acc[2].x);
          red_add_v4(reinterpret_cast<float*>(out_field[1]) + 4 * (size_t)v, acc[0].y, acc[1].y, acc[2].y);
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            atomicAdd(reinterpret_cast<float*>(out_field[0]) + (size_t)c * nv + v, acc[c].x);
            atomicAdd(reinterpret_cast<float*>(out_field[1]) + (size_t)c * nv + v, acc[c].y);
          }
        }
      }
    } else
    {
      const uint32_t d = reinterpret_cast<const uint32_t*>(st + kBlobUnits)[tid];
      const unsigned rem = (d >> 22) & 0xfu;
      T acc[3 * NF];
#pragma unroll
      for (int o = 0; o < 3 * NF; ++o) acc[o] = T(0);
      if (d & 1u) {
        const uint4 codes = reinterpret_cast<const uint4*>(st + kBlobEnt)[tid];
        const unsigned cw[4] = {codes.x, codes.y, codes.z, codes.w};
#pragma unroll
        for (int q = 0; q < kUnitEntries; ++q) {
          const unsigned code = (cw[q >> 1] >> (16 * (q & 1))) & 0xffffu;
          if (code != kEntryNone) {
            const T* p = sob + (size_t)code * NF;
#pragma unroll
            for (int c = 0; c < 3; ++c) add_out<T, NF>(p + c * (TT + 1) * NF, acc + c * NF);
          }
        }
      }
      const unsigned maxrem = __reduce_max_sync(0xffffffffu, rem);
      for (unsigned stp = 1; stp <= maxrem; stp <<= 1) {
#pragma unroll
        for (int o = 0; o < 3 * NF; ++o) {
          const T x = __shfl_down_sync(0xffffffffu, acc[o], stp);
          if (rem >= stp) acc[o] += x;
        }
      }
      if ((d >> 26) & 1u) {
        const int v = reinterpret_cast<const int*>(st + kBlobVtx)[(d >> 14) & 0xffu];
        if constexpr (ORD) {
          T* row = io.part + (size_t)urow * (4 * NF);
#pragma unroll
          for (int f = 0; f < NF; ++f) st_part4(row + 4 * f, acc[f], acc[NF + f], acc[2 * NF + f]);
        } else if constexpr (AOS) {
#pragma unroll
          for (int f = 0; f < NF; ++f)
            red_add_v4(out_field[f] + 4 * (size_t)v, acc[f], acc[NF + f], acc[2 * NF + f]);
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int f = 0; f < NF; ++f) atomicAdd(out_field[f] + (size_t)c * nv + v, acc[c * NF + f]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty_b[sb]);
  }
  return true;
}

}  // namespace ebb
