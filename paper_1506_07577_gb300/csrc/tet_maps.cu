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
//           distinct vertices are gathered once (asynchronously, by a
//           producer warp), per-corner results go to shared memory, and each
//           distinct vertex sums its entries in a fixed order (no
//           shared-memory atomics) and gets one global atomic add per
//           component.
#include <cstdint>

#include "async_copy.cuh"
#include "ebb_internal.h"
#include "tet_io.cuh"
#include "tet_math.cuh"
#include "tet_math_x2.cuh"

namespace ebb {

namespace {

constexpr int kMapThreads = 128;

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

// AOS: vertex-interleaved operands (MapIO::aos): the producer copies each
// vertex's 16 bytes with one cp.async, the reduction adds each vertex's three
// components with one vector atomic.
template <typename T, int MODEL, int OPS, bool AOS>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 4 : 2)
tet_tile_kernel(int ntiles, int nv, const unsigned char* __restrict__ blobs, BlobLayout L,
                const int* __restrict__ perm, T mu0, T lam0, MapIO<T> io, const int* active, int* err,
                int drop_tile, long long wait_cycles) {
  using Z = TileSmem<T, OPS>;
  constexpr int TT = Z::TT, NF = Z::NF, RB = Z::RB, RV = Z::RV;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* ring = smem;
  T* slots = reinterpret_cast<T*>(smem + Z::slot_off(L));
  T* outs = reinterpret_cast<T*>(smem + Z::out_off(L));
  uint64_t* full_b = reinterpret_cast<uint64_t*>(smem + Z::bar_off(L));
  uint64_t* empty_b = full_b + RB;
  uint64_t* full_v = empty_b + RB;
  uint64_t* empty_v = full_v + RV;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty_v + RV);

  if (active != nullptr && *active == 0) return;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int G = gridDim.x;
  if ((int)blockIdx.x >= ntiles) return;
  const int n_my = (ntiles - (int)blockIdx.x + G - 1) / G;
  if (tid == 0) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      mbar_init(&full_b[r], 1);
      mbar_init(&empty_b[r], TT / 32);
    }
#pragma unroll
    for (int r = 0; r < RV; ++r) {
      mbar_init(&full_v[r], 32);
      mbar_init(&empty_v[r], 1);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (tid >= TT) {
    // ---------------------------------------------------------- producer --
    unsigned pend = 0u, pend_parity = 0u;  // blob stages with an unwaited copy
    bool bad = false;
    for (int j = 0; j < n_my + Z::LAG && !bad; ++j) {
      if (j < n_my) {
        const int sb = j % RB;
        bool ok = j < RB || mbar_wait_or_abort(&empty_b[sb], ((j / RB) - 1) & 1u, abort_flag, wait_cycles);
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
          pend_parity = (pend_parity & ~(1u << sb)) | (((unsigned)(j / RB) & 1u) << sb);
        }
      }
      const int jj = j - Z::LAG;
      if (jj >= 0 && jj < n_my) {
        const int sb = jj % RB, sv = jj % RV;
        bool ok = mbar_wait_or_abort(&full_b[sb], (jj / RB) & 1u, abort_flag, wait_cycles);
        if (ok) pend &= ~(1u << sb);
        ok = ok && (jj < RV || mbar_wait_or_abort(&empty_v[sv], ((jj / RV) - 1) & 1u, abort_flag, wait_cycles));
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
    return;
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
    const int sb = j % RB, sv = j % RV;
    const unsigned char* st = ring + (size_t)sb * L.bytes;
    const T* su = slots + (size_t)sv * Z::slot_elems;
    const T* sw = su + 4 * Z::S;
    T* sob = outs + (Z::OB == 2 ? (j & 1) : 0) * Z::out_elems;
    const bool ok = mbar_wait_or_abort(&full_b[sb], (j / RB) & 1u, abort_flag, wait_cycles) &&
                    mbar_wait_or_abort(&full_v[sv], (j / RV) & 1u, abort_flag, wait_cycles);
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
      // The tet's record: Dm^-1, V, mu, lambda in three (FP32) or six (FP64)
      // 16-byte loads.
      T rec[12];
      if constexpr (sizeof(T) == 4) {
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
      return;
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
        if constexpr (AOS) {
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
        if constexpr (AOS) {
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
}

template <typename T, int MODEL, int OPS, bool AOS>
struct TileLaunchCfg {
  static size_t smem;
  static int grid_per_sm;
};
template <typename T, int MODEL, int OPS, bool AOS>
size_t TileLaunchCfg<T, MODEL, OPS, AOS>::smem = 0;
template <typename T, int MODEL, int OPS, bool AOS>
int TileLaunchCfg<T, MODEL, OPS, AOS>::grid_per_sm = 0;

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

template <typename T, int MODEL, int OPS, bool AOS = false>
cudaError_t configure_tiles() {
  cudaError_t e = cudaFuncSetAttribute(tet_tile_kernel<T, MODEL, OPS, AOS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tet_tile_kernel<T, MODEL, OPS, AOS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100);
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

template <typename T, int MODEL, int OPS, bool AOS>
cudaError_t launch_tiles(ebb_rel_s* rel, T mu0, T lam0, const MapIO<T>& io, const int* active,
                         cudaStream_t stream) {
  const Tiles& tl = rel->tiles;
  if (tl.ntiles == 0) return cudaSuccess;
  const BlobLayout& L = layout_of<T>(tl);
  const size_t smem = TileSmem<T, OPS>::bytes(L);
  using Cfg = TileLaunchCfg<T, MODEL, OPS, AOS>;
  if (Cfg::smem != smem) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tet_tile_kernel<T, MODEL, OPS, AOS>,
                                                                  kTileThreads, smem);
    if (e != cudaSuccess) return e;
    Cfg::grid_per_sm = per_sm > 0 ? per_sm : 1;
    Cfg::smem = smem;
  }
  int grid = Cfg::grid_per_sm * sm_count();
  if (grid > tl.ntiles) grid = tl.ntiles;
  const int drop = rel->test_drop_tile;
  tet_tile_kernel<T, MODEL, OPS, AOS><<<grid, kTileThreads, smem, stream>>>(
      tl.ntiles, (int)rel->verts->size, blob_of<T>(tl), L, rel->tet_perm, mu0, lam0, io, active, rel->ctx->d_err,
      drop, drop >= 0 ? kTestWaitCycles : kWaitCycles);
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
