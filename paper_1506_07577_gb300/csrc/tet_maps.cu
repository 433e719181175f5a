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

// ---- tiled: persistent CTAs over tile blobs --------------------------------
// Each CTA walks tiles blockIdx.x, blockIdx.x + G, ... (G = gridDim.x).  The
// integer part of each tile blob (slots, entries, reduction units, vertex
// ids) is fetched with one cp.async.bulk into a 3-deep shared ring, two
// tiles ahead; the per-tet floats (Dm^-1, V, Lame) are read straight from
// the blob in global memory with coalesced loads one tile ahead into
// registers, and the next tile's vertex values are loaded into registers
// while the current tile computes.  Per tile, with one CTA barrier:
//   phase 1  one tet per thread: corner values from the slot vectors,
//            element evaluation, per-corner outputs to shared memory (fields
//            interleaved, conflict-free); then the prefetched vertex values
//            of the next tile go to the other slot buffer;
//                                    -- the one barrier per tile --
//   phase 2  one reduction unit per thread: the sum of at most kUnitEntries
//            entries of one vertex, in a fixed order; the units of one vertex
//            on consecutive lanes are combined by a segmented shuffle tree and
//            the run's first lane issues one atomic add per component (a
//            fire-and-forget reduction).  Every thread does at most
//            kUnitEntries steps, whatever the vertex degrees.
// Slot vectors and per-corner outputs are double buffered, so phase 2 of one
// tile overlaps phase 1 of the next.
// Dynamic shared memory: prefix ring[3] | slot vectors[2] (u[S][4], then
// w[S][4] for K w) | outputs[2][4][3][TT+1][NF] | mbarrier[3].
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz
constexpr int kRing = 3;

template <typename T, int OPS>
struct TileSmem {
  static constexpr bool FO = (OPS & OP_FORCE) != 0;
  static constexpr bool KV = (OPS & OP_KV) != 0;
  static constexpr bool DG = (OPS & OP_DIAG) != 0;
  static constexpr int NF = (FO ? 1 : 0) + (KV ? 1 : 0) + (DG ? 1 : 0);  // output fields
  static constexpr int S = kTileSlots;
  static constexpr int TT = kTileTets;
  static constexpr size_t slot_elems = (size_t)S * 4 * (KV ? 2 : 1);
  static constexpr size_t out_elems = (size_t)4 * 3 * (TT + 1) * NF;  // row TT stays zero
  static constexpr size_t ring_bytes = (size_t)kRing * kBlobPrefix;
  static constexpr size_t bytes = ring_bytes + sizeof(T) * (2 * slot_elems + 2 * out_elems) + kRing * sizeof(uint64_t);
};

template <typename T>
struct TetRegs {
  T B[9];
  T V, mu, lam;
};

// Coalesced loads of one tile's per-tet floats (the blob is zero padded, so
// every thread may load).
template <typename T>
__device__ __forceinline__ void load_tet_regs(const unsigned char* blob, const BlobLayout& L, int tid, T mu0,
                                              T lam0, TetRegs<T>& r) {
  const T* B = reinterpret_cast<const T*>(blob + L.B);
#pragma unroll
  for (int i = 0; i < 9; ++i) r.B[i] = B[i * kTileTets + tid];
  r.V = reinterpret_cast<const T*>(blob + L.V)[tid];
  r.mu = L.mu >= 0 ? reinterpret_cast<const T*>(blob + L.mu)[tid] : mu0;
  r.lam = L.lam >= 0 ? reinterpret_cast<const T*>(blob + L.lam)[tid] : lam0;
}

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
__device__ __forceinline__ void st3(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], 0.f);
}
__device__ __forceinline__ void st3(double* p, const double* v) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  p[2] = v[2];
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

template <typename T, int MODEL, int OPS>
__global__ void __launch_bounds__(kTileTets, sizeof(T) == 4 ? 5 : 2)
tet_tile_kernel(int ntiles, int nv, const unsigned char* __restrict__ blobs, BlobLayout L,
                const int* __restrict__ perm, T mu0, T lam0, MapIO<T> io, const int* active, int* err) {
  using Z = TileSmem<T, OPS>;
  constexpr int TT = Z::TT, NF = Z::NF;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* ring = smem;
  T* slotv = reinterpret_cast<T*>(smem + Z::ring_bytes);
  T* so = slotv + 2 * Z::slot_elems;
  uint64_t* bar = reinterpret_cast<uint64_t*>(so + 2 * Z::out_elems);
  T* out_field[3];
  {
    int f = 0;
    if (Z::FO) out_field[f++] = io.f;
    if (Z::KV) out_field[f++] = io.Kw;
    if (Z::DG) out_field[f++] = io.d;
  }

  if (active != nullptr && *active == 0) return;
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  int tile = blockIdx.x;
  if (tile >= ntiles) return;
  if (tid == 0) {
#pragma unroll
    for (int r = 0; r < kRing; ++r) mbar_init(&bar[r], 1);
    fence_mbar_init();
  }
  // Zero rows (tet index TT) read by padded reduction entries.
  for (int i = tid; i < 2 * 12 * NF; i += TT) {
    const int buf = i / (12 * NF), ac = (i / NF) % 12, f = i % NF;
    so[buf * Z::out_elems + ((size_t)ac * (TT + 1) + TT) * NF + f] = T(0);
  }
  __syncthreads();
  // Ring state, identical in every thread unless a wait times out: bit r of
  // `pend` = a copy into ring slot r is in flight; bit r of `parity` = the
  // phase parity to wait for next.
  unsigned pend = 0u, parity = 0u;
#pragma unroll
  for (int r = 0; r < kRing - 1; ++r) {
    const int t = tile + r * G;
    if (t < ntiles) {
      if (tid == 0) bulk_load(ring + r * kBlobPrefix, blobs + (size_t)t * L.bytes, kBlobPrefix, &bar[r]);
      pend |= 1u << r;
    }
  }
  TetRegs<T> tr;
  load_tet_regs(blobs + (size_t)tile * L.bytes, L, tid, mu0, lam0, tr);
  bool bad = !mbar_wait(&bar[0], 0u, kWaitCycles);
  if (__syncthreads_or(bad)) goto drain;
  pend &= ~1u;
  parity ^= 1u;
  {
    const int4 h = *reinterpret_cast<const int4*>(ring);
    for (int j = tid; j < h.y; j += TT) {
      const int v = reinterpret_cast<const int*>(ring + kBlobVtx)[j];
      T x[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) x[c] = io.u[(size_t)c * nv + v];
      st3(slotv + 4 * j, x);
      if (Z::KV) {
#pragma unroll
        for (int c = 0; c < 3; ++c) x[c] = io.w[(size_t)c * nv + v];
        st3(slotv + 4 * (Z::S + j), x);
      }
    }
  }
  __syncthreads();

  for (int k = 0;; ++k) {
    const int b = k & 1;
    const int rc = k % kRing, rn = (k + 1) % kRing;
    const unsigned char* pre = ring + rc * kBlobPrefix;
    const unsigned char* pren = ring + rn * kBlobPrefix;
    const T* su = slotv + (b ? Z::slot_elems : 0);
    const T* sw = su + 4 * Z::S;
    T* su_next = slotv + (b ? 0 : Z::slot_elems);
    T* sob = so + (b ? Z::out_elems : 0);
    const int next = tile + G;

    // Next tile: wait for its prefix, start loading its vertex values.  No
    // barrier here: a thread whose wait timed out skips the loads that depend
    // on the copy and reports at the tile's barrier below.
    T pu[3], pw[3];
    TetRegs<T> tn;
    int nvu_next = 0;
    bad = false;
    if (next < ntiles) {
      load_tet_regs(blobs + (size_t)next * L.bytes, L, tid, mu0, lam0, tn);
      if (mbar_wait(&bar[rn], (parity >> rn) & 1u, kWaitCycles)) {
        pend &= ~(1u << rn);
        parity ^= 1u << rn;
        nvu_next = reinterpret_cast<const int4*>(pren)->y;
      } else {
        bad = true;
      }
      if (tid < nvu_next) {
        const int v = reinterpret_cast<const int*>(pren + kBlobVtx)[tid];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pu[c] = io.u[(size_t)c * nv + v];
          if (Z::KV) pw[c] = io.w[(size_t)c * nv + v];
        }
      }
    }
    const int4 h = *reinterpret_cast<const int4*>(pre);

    // Phase 1: one tet per thread.
    if (tid < h.x) {
      const uchar4 sl4 = reinterpret_cast<const uchar4*>(pre + kBlobSlots)[tid];
      const int sl[4] = {sl4.x, sl4.y, sl4.z, sl4.w};
      T Du[9], Dw[9];
      {
        T x0[3], xa[3];
        ld3(su + 4 * sl[0], x0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          ld3(su + 4 * sl[j + 1], xa);
#pragma unroll
          for (int c = 0; c < 3; ++c) Du[c * 3 + j] = xa[c] - x0[c];
        }
        if (Z::KV) {
          ld3(sw + 4 * sl[0], x0);
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            ld3(sw + 4 * sl[j + 1], xa);
#pragma unroll
            for (int c = 0; c < 3; ++c) Dw[c * 3 + j] = xa[c] - x0[c];
          }
        }
      }
      T fo[4][3], ko[4][3], dgo[4][3];
      const bool ok = element_eval<T, MODEL, OPS>(tr.B, tr.V, tr.mu, tr.lam, Du, Dw, fo, ko, dgo);
      if (!ok) raise_error(err, EBB_ERR_INVERTED, perm[h.z + tid]);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T v[NF > 0 ? NF : 1];
          int f = 0;
          if (Z::FO) v[f++] = ok ? fo[a][c] : T(0);
          if (Z::KV) v[f++] = ok ? ko[a][c] : T(0);
          if (Z::DG) v[f++] = ok ? dgo[a][c] : T(0);
          st_out<T, NF>(sob + ((size_t)(a * 3 + c) * (TT + 1) + tid) * NF, v);
        }
      }
    }
    if (tid < nvu_next) {
      st3(su_next + 4 * tid, pu);
      if (Z::KV) st3(su_next + 4 * (Z::S + tid), pw);
    }
    if (__syncthreads_or(bad)) goto drain;

    // Ring slot of tile k-1 is free (its phase 2 finished before the barrier):
    // refill it with the tile kRing-1 ahead.
    {
      const int tf = tile + (kRing - 1) * G;
      if (tf < ntiles) {
        const int rf = (k + kRing - 1) % kRing;
        if (tid == 0) {
          fence_proxy_async_smem();
          bulk_load(ring + rf * kBlobPrefix, blobs + (size_t)tf * L.bytes, kBlobPrefix, &bar[rf]);
        }
        pend |= 1u << rf;
      }
    }

    // Phase 2: one reduction unit per thread: kUnitEntries independent loads.
    {
      const uint32_t d = reinterpret_cast<const uint32_t*>(pre + kBlobUnits)[tid];
      const unsigned rem = (d >> 22) & 0xfu;
      T acc[3 * NF];
#pragma unroll
      for (int o = 0; o < 3 * NF; ++o) acc[o] = T(0);
      if (d & 1u) {
        const uint4 codes = reinterpret_cast<const uint4*>(pre + kBlobEnt)[tid];
        const unsigned cw[4] = {codes.x, codes.y, codes.z, codes.w};
#pragma unroll
        for (int q = 0; q < kUnitEntries; ++q) {
          const unsigned code = (cw[q >> 1] >> (16 * (q & 1))) & 0xffffu;
          const int base = (int)(code >> 8) * 3 * (TT + 1) + (int)(code & 255u);
#pragma unroll
          for (int c = 0; c < 3; ++c) add_out<T, NF>(sob + ((size_t)base + c * (TT + 1)) * NF, acc + c * NF);
        }
      }
      const unsigned maxrem = __reduce_max_sync(0xffffffffu, rem);
      for (unsigned st = 1; st <= maxrem; st <<= 1) {
#pragma unroll
        for (int o = 0; o < 3 * NF; ++o) {
          const T x = __shfl_down_sync(0xffffffffu, acc[o], st);
          if (rem >= st) acc[o] += x;
        }
      }
      if ((d >> 26) & 1u) {
        const int v = reinterpret_cast<const int*>(pre + kBlobVtx)[(d >> 14) & 0xffu];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int f = 0; f < NF; ++f) atomicAdd(out_field[f] + (size_t)c * nv + v, acc[c * NF + f]);
      }
    }
    tr = tn;
    if (next >= ntiles) break;
    tile = next;
  }
  return;

drain:
  // A copy did not complete in time: report it and wait (bounded) for the
  // copies still in flight before the CTA's shared memory goes away.
  if (tid == 0) raise_error(err, EBB_ERR_TIMEOUT, blockIdx.x);
#pragma unroll
  for (int r = 0; r < kRing; ++r)
    if ((pend >> r) & 1u) mbar_wait(&bar[r], (parity >> r) & 1u, kWaitCycles);
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
  const size_t smem = TileSmem<T, OPS>::bytes;
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
