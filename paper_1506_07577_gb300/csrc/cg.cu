// Linearised backward-Euler step with a Jacobi-preconditioned CG solve.
//
// Section 7.2: per time step the elastic forces and stiffness are evaluated,
// a linear system is built and solved for the vertex velocities with a
// Jacobi-preconditioned conjugate gradient solver written as data-parallel
// kernels; Section 7.3 reuses the same integrator and solver.  The system is
//   A = M + dt^2 K(x_n),   b = dt (f(x_n) + M g - dt K(x_n) v_n)
// with pinned rows and columns removed, solved from dv = 0; then
// v += dv, u += dt v.
//
// Global reductions (dot products) follow the two-pass scheme of Section 6.2
// "Reductions": the first pass is fused into the kernel producing the values
// (per-block partial sums); the second pass is done by the last block of the
// same kernel to finish, which sums the partials in block order (so the
// result is deterministic) and updates the CG scalars on the device.
// Scalars never leave the device inside the loop; the host reads one status
// word per batch of iterations.  CG vectors, dots and updates are FP64 in
// both precisions; the element maps run in the element precision T.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "ebb_internal.h"

namespace ebb {

namespace {

constexpr int kVecThreads = 256;
constexpr int kVecBlocks = 4 * 152;   // 4 blocks per SM on a 152-SM GB300
constexpr int kChunk = 8;             // CG iterations launched between host status reads (even)

// Device-side CG state.  `count` are the arrival counters of the three
// reduction sites (init, p.Ap, r.z); the last block of a kernel resets its own.
struct CgScalars {
  double rz[2];      // r.z, indexed by iteration parity
  double rr;         // r.r after the last update
  double bb;         // b.b
  double alpha, beta;
  int active[2];     // iteration with parity s runs iff active[s]
  int iter;          // iterations completed
  int status;        // EBB_OK, EBB_ERR_CG_BREAKDOWN or EBB_ERR_TIMEOUT
  unsigned count[3];
  unsigned bar_count, bar_gen;   // grid barrier of the fused iteration kernel
};

template <typename PT>
__device__ __forceinline__ bool is_pinned(const PT* pin, int v) {
  return pin != nullptr && pin[v] != 0;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block sum of two values; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kVecThreads / 32], sb[kVecThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = l < kVecThreads / 32 ? sa[l] : 0.0;
    b = l < kVecThreads / 32 ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
  __syncthreads();
}

// Two-pass global sum of (a, b) (Section 6.2 "Reductions"): every block
// writes its partial; the last block to arrive sums all partials in block
// order -- the same order every time, so the result is deterministic -- and
// returns true with the totals in (a, b) for all of its threads.
__device__ __forceinline__ bool reduce_last(double& a, double& b, double* part, unsigned* counter) {
  __shared__ unsigned s_last;
  __shared__ double ra, rb;
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
    __threadfence();
    s_last = atomicAdd(counter, 1u) == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kVecThreads) {
    x += __ldcg(part + 2 * i);
    y += __ldcg(part + 2 * i + 1);
  }
  block_sum2(x, y);
  if (threadIdx.x == 0) {
    ra = x;
    rb = y;
    *counter = 0u;
  }
  __syncthreads();
  a = ra;
  b = rb;
  return true;
}

// Element-precision operands of the step's maps are library-internal, so in
// FP32 they are stored vertex-interleaved (AOS: nv groups of x, y, z,
// padding), which lets the maps fetch a vertex with one 16-byte copy and add
// into it with one vector atomic.
template <bool AOS>
__device__ __forceinline__ size_t vidx(int nv, int v, int k) {
  return AOS ? 4 * (size_t)v + k : (size_t)k * nv + v;
}

// ue = u, ve = v in the element precision (mixed only); accumulators zeroed.
template <typename T, bool AOS>
__global__ void step_prep_kernel(int nv, const double* __restrict__ u, const double* __restrict__ v, T* ue,
                                 T* ve, T* acc_f, T* acc_kv, T* acc_d, T* acc_kp, bool copy) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nv; x += gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < (AOS ? 4 : 3); ++k) {
      const size_t i = vidx<AOS>(nv, x, k);
      if (copy) {
        ue[i] = k < 3 ? (T)u[(size_t)k * nv + x] : T(0);
        ve[i] = k < 3 ? (T)v[(size_t)k * nv + x] : T(0);
      }
      acc_f[i] = T(0);
      acc_kv[i] = T(0);
      acc_d[i] = T(0);
      acc_kp[i] = T(0);
    }
  }
}

// Lumped mass m_v = sum over (tet, corner) entries of v of rho V_t / 4,
// gathered through the vertex -> (tet, corner) index in a fixed order so the
// result does not depend on thread scheduling.
__global__ void mass_kernel(int nv, const int* __restrict__ off, const int* __restrict__ ent,
                            const double* __restrict__ V, double rho, double* m) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int e = off[v]; e < off[v + 1]; ++e) s += V[ent[e] >> 2];
  m[v] = 0.25 * rho * s;
}

struct StepConst {
  int nv;
  double dt;
  double g[3];
  double rtol;
  int max_iters;
};

// b = dt (f + m g - dt K v) (0 on pinned rows); r = b; z = r / diag(A);
// p = z; y = 0; then r.z and r.r, and the CG state for iteration 0.
template <typename T, typename PT, bool AOS>
__global__ void __launch_bounds__(kVecThreads)
cg_init_kernel(StepConst c, const PT* __restrict__ pin, const double* __restrict__ mass,
               const T* __restrict__ acc_f, const T* __restrict__ acc_kv, const T* __restrict__ acc_d,
               double* r, double* p, double* y, double* dinv, T* pe, double* part, CgScalars* sc) {
  const int n = 3 * c.nv;
  double rz = 0.0, rr = 0.0;
#pragma unroll 4
  for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += kVecBlocks * kVecThreads) {
    const int comp = i >= c.nv ? (i >= 2 * c.nv ? 2 : 1) : 0;
    const int vtx = i - comp * c.nv;
    const size_t ie = vidx<AOS>(c.nv, vtx, comp);
    double b = 0.0, di = 1.0;
    if (!is_pinned(pin, vtx)) {
      const double m = mass[vtx];
      b = c.dt * ((double)acc_f[ie] + m * c.g[comp] - c.dt * (double)acc_kv[ie]);
      di = 1.0 / (m + c.dt * c.dt * (double)acc_d[ie]);
    }
    const double z = b * di;
    r[i] = b;
    p[i] = z;
    y[i] = 0.0;
    dinv[i] = di;
    if (pe) pe[ie] = (T)z;
    rz += b * z;
    rr += b * b;
  }
  if (reduce_last(rz, rr, part, &sc->count[0]) && threadIdx.x == 0) {
    sc->rz[0] = rz;
    sc->rz[1] = 0.0;
    sc->rr = rr;
    sc->bb = rr;
    sc->alpha = sc->beta = 0.0;
    sc->iter = 0;
    sc->status = EBB_OK;
    sc->active[0] = (c.max_iters > 0 && sqrt(rr) > c.rtol * sqrt(rr)) ? 1 : 0;
    sc->active[1] = 0;
  }
}

// Grid-wide barrier of a cooperative launch (every block co-resident).  The
// last block to arrive resets the counter and advances the generation the
// others spin on.  Bounded: returns false if the barrier did not complete
// within `limit` SM cycles.
__device__ bool grid_sync(unsigned* count, unsigned* gen, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = gen;
    const unsigned g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      *count = 0u;
      __threadfence();
      atomicExch(gen, g + 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > limit) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// FP64 is slow on GB300, so the iteration kernel's reductions keep FP64 adds
// few: values go through shared memory and one warp adds them (kVecThreads/32
// per lane, then a 5-level shuffle tree), instead of a shuffle tree in every
// warp.  Block sum of (a, b), fixed order; result in thread 0.
__device__ __forceinline__ void block_sum2_w0(double& a, double& b) {
  __shared__ double sa[kVecThreads], sb[kVecThreads];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = 0.0, y = 0.0;
#pragma unroll
    for (int i = 0; i < kVecThreads / 32; ++i) {
      x += sa[threadIdx.x + 32 * i];
      y += sb[threadIdx.x + 32 * i];
    }
    a = warp_sum(x);
    b = warp_sum(y);
  }
  __syncthreads();
}

// Sums of part[stride*i + 0] and part[stride*i + 1] (the latter only when
// stride is 2) over i < n, in a fixed order, by warp 0: the same in every
// block, so every block obtains the same values.  Result in lane 0 of warp 0.
__device__ __forceinline__ void sum_partials_w0(const double* part, int n, int stride, double& a, double& b) {
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < n; i += 32) {
    x += __ldcg(part + (size_t)stride * i);
    if (stride == 2) y += __ldcg(part + (size_t)stride * i + 1);
  }
  a = warp_sum(x);
  b = warp_sum(y);
}

constexpr long long kGridWaitCycles = 2000000000LL;  // about 1 s at 2 GHz

// dt^2 times a K p entry, in FP64: in the element precision first when that
// is FP32 (K p carries FP32 accuracy either way), saving an FP64 multiply.
__device__ __forceinline__ double dt2_times(float kp, double dt2) { return (double)((float)dt2 * kp); }
__device__ __forceinline__ double dt2_times(double kp, double dt2) { return dt2 * kp; }

// One CG iteration after the K p map, in one cooperative launch (the three
// vector passes of the iteration separated by grid barriers, instead of
// three launches with last-block reductions):
//   A  q = Ap = M p + dt^2 K p (kept in qz); p.Ap    -> alpha = r.z / p.Ap
//   B  y += alpha p; r -= alpha q; z = r / diag A (kept in qz); r.z, r.r
//                                                      -> beta, next active
//   C  p = z + beta p; K p accumulator cleared
// On GB300 FP64 arithmetic runs at a small fraction of the FP32 rate and
// bounds these passes, so each FP64 quantity is formed once (about eight
// FP64 operations per free row and iteration) and q, z go through memory.
// Each pass walks vertices (grid-stride, the same vertices per thread in
// every pass), loading all three components at once; pinned rows keep
// r = p = 0 and are skipped.  Every block sums the per-block partials of a
// pass in the same fixed order (deterministic, identical in every block);
// block 0 publishes the scalars.  A barrier that does not complete sets
// EBB_ERR_TIMEOUT in the CG status.
template <typename T, typename PT, bool AOS>
__global__ void __launch_bounds__(kVecThreads)
cg_iter_kernel(StepConst c, int s, const PT* __restrict__ pin, const double* __restrict__ mass,
               double* __restrict__ p, T* __restrict__ acc_kp, const double* __restrict__ dinv,
               double* __restrict__ r, double* __restrict__ y, double* __restrict__ qz, T* __restrict__ pe,
               double* __restrict__ part_a, double* __restrict__ part_b, CgScalars* sc) {
  if (!sc->active[s] || sc->status != EBB_OK) {
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->active[s ^ 1] = 0;
    return;
  }
  const int nv = c.nv;
  const int stride = gridDim.x * kVecThreads;
  const int v0 = blockIdx.x * kVecThreads + threadIdx.x;
  const double dt2 = c.dt * c.dt;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;

  // A: q = Ap and p.Ap
  double pq = 0.0, zero = 0.0;
  for (int v = v0; v < nv; v += stride) {
    if (is_pinned(pin, v)) continue;
    const double m = mass[v];
    double pv[3];
    T kv[3];
    if constexpr (AOS) {
      const float4 k4 = reinterpret_cast<const float4*>(acc_kp)[v];
      kv[0] = k4.x;
      kv[1] = k4.y;
      kv[2] = k4.z;
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) kv[k] = acc_kp[(size_t)k * nv + v];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) pv[k] = p[(size_t)k * nv + v];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double q = fma(m, pv[k], dt2_times(kv[k], dt2));
      qz[(size_t)k * nv + v] = q;
      pq = fma(pv[k], q, pq);
    }
  }
  __shared__ double s_scal[2];
  block_sum2_w0(pq, zero);
  if (threadIdx.x == 0) part_a[blockIdx.x] = pq;
  if (!grid_sync(&sc->bar_count, &sc->bar_gen, kGridWaitCycles)) {
    if (threadIdx.x == 0) atomicCAS(&sc->status, EBB_OK, EBB_ERR_TIMEOUT);
    return;
  }
  const double rz_old = sc->rz[s];
  if (threadIdx.x < 32) {
    sum_partials_w0(part_a, gridDim.x, 1, pq, zero);
    if (threadIdx.x == 0) {
      s_scal[0] = pq;
      s_scal[1] = pq > 0.0 ? rz_old / pq : 0.0;
    }
  }
  __syncthreads();
  pq = s_scal[0];
  const double alpha = s_scal[1];
  if (!(pq > 0.0)) {
    if (lead) {
      sc->alpha = 0.0;
      sc->status = EBB_ERR_CG_BREAKDOWN;
      sc->active[s ^ 1] = 0;
    }
    return;
  }
  if (lead) sc->alpha = alpha;

  // B: y, r, z and the dots r.z, r.r
  double rz = 0.0, rr = 0.0;
  for (int v = v0; v < nv; v += stride) {
    if (is_pinned(pin, v)) continue;
    double pv[3], qv[3], rv[3], yv[3], dv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const size_t i = (size_t)k * nv + v;
      pv[k] = p[i];
      qv[k] = qz[i];
      rv[k] = r[i];
      yv[k] = y[i];
      dv[k] = dinv[i];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const size_t i = (size_t)k * nv + v;
      y[i] = fma(alpha, pv[k], yv[k]);
      const double ri = fma(-alpha, qv[k], rv[k]);
      const double zi = ri * dv[k];
      r[i] = ri;
      qz[i] = zi;
      rz = fma(ri, zi, rz);
      rr = fma(ri, ri, rr);
    }
  }
  block_sum2_w0(rz, rr);
  if (threadIdx.x == 0) {
    part_b[2 * blockIdx.x] = rz;
    part_b[2 * blockIdx.x + 1] = rr;
  }
  if (!grid_sync(&sc->bar_count, &sc->bar_gen, kGridWaitCycles)) {
    if (threadIdx.x == 0) atomicCAS(&sc->status, EBB_OK, EBB_ERR_TIMEOUT);
    return;
  }
  __shared__ double s_beta;
  if (threadIdx.x < 32) {
    sum_partials_w0(part_b, gridDim.x, 2, rz, rr);
    if (threadIdx.x == 0) s_beta = rz / rz_old;
  }
  __syncthreads();
  const double beta = s_beta;
  if (lead) {
    const int it = sc->iter + 1;
    sc->iter = it;
    sc->beta = beta;
    sc->rz[s ^ 1] = rz;
    sc->rr = rr;
    sc->active[s ^ 1] = (it < c.max_iters && sqrt(rr) > c.rtol * sqrt(sc->bb)) ? 1 : 0;
  }

  // C: p = z + beta p
  for (int v = v0; v < nv; v += stride) {
    const bool pinned = is_pinned(pin, v);
    double zv[3], pv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const size_t i = (size_t)k * nv + v;
      zv[k] = pinned ? 0.0 : qz[i];
      pv[k] = pinned ? 0.0 : p[i];
    }
    double pn[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      pn[k] = pinned ? 0.0 : fma(beta, pv[k], zv[k]);
      p[(size_t)k * nv + v] = pn[k];
    }
    if constexpr (AOS) {
      if (pe) reinterpret_cast<float4*>(pe)[v] = make_float4((float)pn[0], (float)pn[1], (float)pn[2], 0.f);
      reinterpret_cast<float4*>(acc_kp)[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (pe) pe[(size_t)k * nv + v] = (T)pn[k];
        acc_kp[(size_t)k * nv + v] = T(0);
      }
    }
  }
}

// Blocks of cg_iter_kernel: all co-resident (a cooperative launch), at most
// kVecBlocks (the size of the partial-sum arrays).
template <typename T, typename PT, bool AOS>
int iter_grid() {
  static int g = 0;
  if (g == 0) {
    int per_sm = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_iter_kernel<T, PT, AOS>, kVecThreads, 0);
    g = std::min(kVecBlocks, std::min(per_sm, 2) * std::max(nsm, 1));
    if (g < 1) g = 1;
  }
  return g;
}

template <typename T, typename PT, bool AOS>
cudaError_t launch_cg_iter(int grid, cudaStream_t st, StepConst c, int s, const PT* pin, const double* mass,
                           double* p, T* acc_kp, const double* dinv, double* r, double* y, double* qz, T* pe,
                           double* part_a, double* part_b, CgScalars* sc) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kVecThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cg_iter_kernel<T, PT, AOS>, c, s, pin, mass, p, acc_kp, dinv, r, y, qz, pe, part_a,
                            part_b, sc);
}

// Adjoint solve set-up: b = dL/dv' + dt dL/du' (0 on pinned rows); r = b;
// z = r / diag(A) (diag from the forward solve at the same state); p = z;
// y = 0; r.z, r.r and the CG state for iteration 0.
template <typename PT>
__global__ void __launch_bounds__(kVecThreads)
cg_init_rhs_kernel(StepConst c, const PT* __restrict__ pin, const double* __restrict__ gu,
                   const double* __restrict__ gv, const double* __restrict__ dinv, double* r, double* p, double* y,
                   double* part, CgScalars* sc) {
  const int n = 3 * c.nv;
  double rz = 0.0, rr = 0.0;
#pragma unroll 4
  for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += kVecBlocks * kVecThreads) {
    const int comp = i >= c.nv ? (i >= 2 * c.nv ? 2 : 1) : 0;
    const int vtx = i - comp * c.nv;
    const double b = is_pinned(pin, vtx) ? 0.0 : gv[i] + c.dt * gu[i];
    const double z = b * dinv[i];
    r[i] = b;
    p[i] = z;
    y[i] = 0.0;
    rz += b * z;
    rr += b * b;
  }
  if (reduce_last(rz, rr, part, &sc->count[0]) && threadIdx.x == 0) {
    sc->rz[0] = rz;
    sc->rz[1] = 0.0;
    sc->rr = rr;
    sc->bb = rr;
    sc->alpha = sc->beta = 0.0;
    sc->iter = 0;
    sc->status = EBB_OK;
    sc->active[0] = (c.max_iters > 0 && sqrt(rr) > c.rtol * sqrt(rr)) ? 1 : 0;
    sc->active[1] = 0;
  }
}

// w = v' = v + dv; adjoint accumulators zeroed.
__global__ void vjp_prep_kernel(int n, const double* __restrict__ v, const double* __restrict__ dv, double* w,
                                double* acc_kl, double* acc_xq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    w[i] = v[i] + dv[i];
    acc_kl[i] = 0.0;
    acc_xq[i] = 0.0;
  }
}

// dL/du = gu - dt K lam - dt^2 d/dx[lam^T K v'];  dL/dv = gv + dt gu - dt^2 K lam.
__global__ void vjp_finish_kernel(int n, double dt, const double* __restrict__ acc_kl,
                                  const double* __restrict__ acc_xq, double* gu, double* gv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double g = gu[i], kl = acc_kl[i];
    gu[i] = g - dt * kl - dt * dt * acc_xq[i];
    gv[i] = gv[i] + dt * g - dt * dt * kl;
  }
}

// dv = v' - v (a step whose new velocity the caller already holds).
__global__ void vel_diff_kernel(int n, const double* __restrict__ v_next, const double* __restrict__ v, double* dv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dv[i] = v_next[i] - v[i];
}

// v += dv; u += dt v.
__global__ void step_finish_kernel(int n, double dt, const double* __restrict__ y, double* u, double* v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double vi = v[i] + y[i];
    v[i] = vi;
    u[i] += dt * vi;
  }
}

}  // namespace

// Everything a captured CG chunk bakes into its kernel arguments; a change
// of any field re-captures the graph.
struct ChunkKey {
  int elem_bytes, pin_bytes, model, reduce, assembled;
  unsigned layout_gen;  // tile blobs baked into the captured map launches
  double mu0, lam0;
  StepConst c;
  const void* pin;
  const void* u;
};

struct StepScratch {
  int nv = 0;
  cudaStream_t stream = nullptr;        // internal stream (capturable)
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t chunk = nullptr;      // kChunk captured CG iterations
  ChunkKey key;
  bool have_key = false;
  void* acc[4] = {nullptr, nullptr, nullptr, nullptr};   // f, Kv, diag, Kp in element precision
  void* ue = nullptr;                                    // element-precision displacement
  void* pe = nullptr;                                    // element-precision v, then p
  double *r = nullptr, *p = nullptr, *y = nullptr, *dinv = nullptr, *mass = nullptr;
  double* qz = nullptr;     // Ap, then z = r / diag A, within one CG iteration
  double* part = nullptr;   // 2 sets of kVecBlocks pairs
  CgScalars* sc = nullptr;
  CgScalars* h_sc = nullptr;
  double rho = -1.0;
  double *vjp_w = nullptr, *vjp_kl = nullptr, *vjp_xq = nullptr;   // adjoint-only buffers
  double *u_int = nullptr, *v_int = nullptr;                        // state in the internal vertex order
  unsigned char* pin_int = nullptr;
};

void free_step_scratch(ebb_rel_s* rel) {
  StepScratch* s = rel->step;
  if (!s) return;
  for (void* a : s->acc) cudaFree(a);
  cudaFree(s->ue);
  cudaFree(s->pe);
  cudaFree(s->r);
  cudaFree(s->p);
  cudaFree(s->y);
  cudaFree(s->dinv);
  cudaFree(s->qz);
  cudaFree(s->mass);
  cudaFree(s->part);
  cudaFree(s->sc);
  if (s->h_sc) cudaFreeHost(s->h_sc);
  cudaFree(s->vjp_w);
  cudaFree(s->vjp_kl);
  cudaFree(s->vjp_xq);
  cudaFree(s->u_int);
  cudaFree(s->v_int);
  cudaFree(s->pin_int);
  if (s->chunk) cudaGraphExecDestroy(s->chunk);
  if (s->ev) cudaEventDestroy(s->ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  rel->step = nullptr;
}

namespace {

struct VjpArgs {
  double* gu;     // in: dL/du', out: dL/du
  double* gv;     // in: dL/dv', out: dL/dv
  double* gmu;    // per-tet dL/dmu (+=), caller's tet order, may be null
  double* glam;   // per-tet dL/dlambda (+=), may be null
  const double* v_next;  // the step's new velocity when the caller has it (no forward solve), else null
};

ebb_status_t ensure_scratch(ebb_ctx_s* ctx, ebb_rel_s* tets) {
  const int nv = (int)tets->verts->size;
  if (tets->step && tets->step->nv == nv) return EBB_OK;
  free_step_scratch(tets);
  StepScratch* s = new StepScratch();
  tets->step = s;
  s->nv = nv;
  const size_t n = (size_t)3 * nv;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMalloc(&s->acc[i], n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->ue, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->pe, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->r, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->p, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->y, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->dinv, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->qz, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->mass, (size_t)nv * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->part, 4 * kVecBlocks * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->sc, sizeof(CgScalars));
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_sc, sizeof(CgScalars));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_step_scratch(tets);
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, "device allocation for implicit-step scratch failed");
  }
  return EBB_OK;
}

template <typename T, typename PT>
ebb_status_t step_impl(ebb_ctx_s* ctx, ebb_rel_s* tets, double* u, double* v, const PT* pin,
                       const ebb_step_params_t* prm, ebb_cg_report_t* rep, const VjpArgs* vjp = nullptr) {
  const bool mixed = sizeof(T) == 4;
  StepScratch* s = tets->step;
  const int nv = s->nv;
  const int n = 3 * nv;
  // All step work runs on the library's own stream, ordered after the
  // caller's stream; the call is synchronous.
  cudaStream_t st = s->stream;
  cudaError_t e = cudaEventRecord(s->ev, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, s->ev, 0);
  if (e != cudaSuccess) return cuda_check(ctx, e, "ordering after the caller's stream");
  T* acc_f = (T*)s->acc[0];
  T* acc_kv = (T*)s->acc[1];
  T* acc_d = (T*)s->acc[2];
  T* acc_kp = (T*)s->acc[3];
  T* ue = (T*)s->ue;
  T* pe = (T*)s->pe;

  if (tets->vindex.off == nullptr) return set_error(ctx, EBB_ERR_STATE, "relation has no vertex index");
  if (s->rho != prm->rho) {
    mass_kernel<<<(nv + 255) / 256, 256, 0, st>>>(nv, tets->vindex.off, tets->vindex.ent, tets->s64.V, prm->rho,
                                                   s->mass);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(ctx, e, "lumped mass");
    s->rho = prm->rho;
  }

  StepConst c;
  memset(&c, 0, sizeof c);
  c.nv = nv;
  c.dt = prm->dt;
  c.g[0] = prm->gravity[0];
  c.g[1] = prm->gravity[1];
  c.g[2] = prm->gravity[2];
  c.rtol = prm->rtol;
  c.max_iters = prm->max_iters;

  const int vgrid = 4 * 152;
  // Arrival counters of the last-block reductions start at zero.
  e = cudaMemsetAsync(s->sc, 0, sizeof(CgScalars), st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "CG state reset");
  // FP32 operands are vertex-interleaved (see vidx).
  bool aos = false;
  if constexpr (sizeof(T) == 4) aos = mixed;   // every reduction variant takes interleaved operands
  if (aos)
    step_prep_kernel<T, true><<<vgrid, 256, 0, st>>>(nv, u, v, ue, pe, acc_f, acc_kv, acc_d, acc_kp, mixed);
  else
    step_prep_kernel<T, false><<<vgrid, 256, 0, st>>>(nv, u, v, ue, pe, acc_f, acc_kv, acc_d, acc_kp, mixed);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(ctx, e, "step prep");

  const T mu0 = (T)prm->mu, lam0 = (T)prm->lambda;
  MapIO<T> io;
  io.u = mixed ? ue : (const T*)u;
  io.w = mixed ? pe : (const T*)v;
  io.f = acc_f;
  io.Kw = acc_kv;
  io.d = acc_d;
  io.aos = aos;
  e = launch_tet_map<T>(tets, prm->model, OP_FORCE | OP_KV | OP_DIAG, prm->reduce, mu0, lam0, io, nullptr, st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "force/Kv/diag map");
  // EBB_STEP_ASSEMBLED: K(x_n) on the edge relation, once per step; the CG
  // products below read it instead of re-evaluating the elements.
  const bool assembled = (prm->flags & EBB_STEP_ASSEMBLED) != 0;
  if (assembled) {
    e = launch_assemble<T>(tets, prm->model, mu0, lam0, io, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "stiffness assembly");
  }

  double* part_a = s->part;
  double* part_b = s->part + 2 * kVecBlocks;
  if (aos)
    cg_init_kernel<T, PT, true><<<kVecBlocks, kVecThreads, 0, st>>>(c, pin, s->mass, acc_f, acc_kv, acc_d, s->r,
                                                                     s->p, s->y, s->dinv, pe, part_a, s->sc);
  else
    cg_init_kernel<T, PT, false><<<kVecBlocks, kVecThreads, 0, st>>>(c, pin, s->mass, acc_f, acc_kv, acc_d, s->r,
                                                                      s->p, s->y, s->dinv, mixed ? pe : nullptr,
                                                                      part_a, s->sc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(ctx, e, "CG init");

  MapIO<T> kio;
  kio.u = io.u;
  kio.w = mixed ? pe : (const T*)s->p;
  kio.Kw = acc_kp;
  kio.aos = aos;

  // kChunk CG iterations (plus the status read-back) are captured once as a
  // CUDA graph and relaunched until the device reports convergence.
  ChunkKey key;
  memset(&key, 0, sizeof key);
  key.elem_bytes = (int)sizeof(T);
  key.pin_bytes = (int)sizeof(PT);
  key.model = prm->model;
  key.reduce = prm->reduce;
  key.assembled = assembled ? 1 : 0;
  key.layout_gen = tets->layout_gen;
  key.mu0 = prm->mu;
  key.lam0 = prm->lambda;
  key.c = c;
  key.pin = pin;
  key.u = kio.u;
  if (!s->chunk || !s->have_key || memcmp(&key, &s->key, sizeof key) != 0) {
    if (s->chunk) cudaGraphExecDestroy(s->chunk);
    s->chunk = nullptr;
    s->have_key = false;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_check(ctx, e, "CG chunk capture");
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < kChunk && le == cudaSuccess; ++k) {
      const int par = k & 1;
      le = assembled ? launch_spmv<T>(tets, kio.w, acc_kp, aos, &s->sc->active[par], st)
                     : launch_tet_map<T>(tets, prm->model, OP_KV, prm->reduce, mu0, lam0, kio, &s->sc->active[par], st);
      if (le == cudaSuccess)
        le = aos ? launch_cg_iter<T, PT, true>(iter_grid<T, PT, true>(), st, c, par, pin, s->mass, s->p, acc_kp,
                                               s->dinv, s->r, s->y, s->qz, pe, part_a, part_b, s->sc)
                 : launch_cg_iter<T, PT, false>(iter_grid<T, PT, false>(), st, c, par, pin, s->mass, s->p, acc_kp,
                                                s->dinv, s->r, s->y, s->qz, mixed ? pe : nullptr, part_a, part_b,
                                                s->sc);
    }
    if (le == cudaSuccess) le = cudaMemcpyAsync(s->h_sc, s->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_check(ctx, le != cudaSuccess ? le : e, "CG chunk capture");
    }
    e = cudaGraphInstantiate(&s->chunk, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      s->chunk = nullptr;
      return cuda_check(ctx, e, "CG chunk instantiate");
    }
    s->key = key;
    s->have_key = true;
  }

  ebb_status_t status = EBB_OK;
  auto run_chunks = [&]() -> cudaError_t {
    int launched = 0;
    while (true) {
      cudaError_t ce2 = cudaGraphLaunch(s->chunk, st);
      if (ce2 == cudaSuccess) ce2 = cudaStreamSynchronize(st);
      if (ce2 != cudaSuccess) return ce2;
      launched += kChunk;
      const CgScalars& h = *s->h_sc;
      if (h.status != EBB_OK) {
        status = h.status;
        return cudaSuccess;
      }
      if (!h.active[h.iter & 1] || h.iter >= prm->max_iters) return cudaSuccess;
      if (launched > prm->max_iters + 2 * kChunk) return cudaSuccess;  // defensive bound
    }
  };
  if (vjp != nullptr && vjp->v_next != nullptr) {
    // The caller holds the step's new velocity (a forward replay): dv = v' - v
    // replaces the forward solve.
    vel_diff_kernel<<<vgrid, 256, 0, st>>>(n, vjp->v_next, v, s->y);
    e = cudaGetLastError();
  } else {
    e = run_chunks();
  }
  if (e != cudaSuccess) return cuda_check(ctx, e, "CG chunk");

  if (vjp != nullptr) {
    // Adjoint of the step just solved (FP64, StVK): v' = v + dv, then the
    // adjoint solve A lam = gv + dt gu with the same operator (the captured
    // iterations act on p, K p and the forward state), then the adjoint map.
    if (status != EBB_OK) return set_error(ctx, status, "forward solve failed inside the step VJP");
    vjp_prep_kernel<<<vgrid, 256, 0, st>>>(n, v, s->y, s->vjp_w, s->vjp_kl, s->vjp_xq);
    cg_init_rhs_kernel<PT><<<kVecBlocks, kVecThreads, 0, st>>>(c, pin, vjp->gu, vjp->gv, s->dinv, s->r, s->p, s->y,
                                                              part_a, s->sc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = run_chunks();
    if (e != cudaSuccess) return cuda_check(ctx, e, "adjoint solve");
    e = launch_adjoint_map(tets, prm->mu, prm->lambda, u, s->y, s->vjp_w, s->vjp_kl, s->vjp_xq, vjp->gmu, vjp->glam,
                           prm->dt, st);
    if (e == cudaSuccess) {
      vjp_finish_kernel<<<vgrid, 256, 0, st>>>(n, prm->dt, s->vjp_kl, s->vjp_xq, vjp->gu, vjp->gv);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_check(ctx, e, "adjoint map");
  } else {
    step_finish_kernel<<<vgrid, 256, 0, st>>>(n, prm->dt, s->y, u, v);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_sc, s->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "step finish");
  const CgScalars& h = *s->h_sc;
  const double rel = h.bb > 0.0 ? std::sqrt(h.rr / h.bb) : 0.0;
  if (rep) {
    rep->iters = h.iter;
    rep->rel_residual = rel;
  }
  // Device-raised errors (inverted elements) take precedence.
  cudaError_t ce = cudaMemcpyAsync(ctx->h_err, ctx->d_err, ERRW_WORDS * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_check(ctx, ce, "status read");
  if (ctx->h_err[ERRW_CODE] != 0) {
    const int code = ctx->h_err[ERRW_CODE], idx = ctx->h_err[ERRW_INDEX];
    cudaMemsetAsync(ctx->d_err, 0, ERRW_WORDS * sizeof(int), st);
    cudaStreamSynchronize(st);
    char buf[128];
    snprintf(buf, sizeof buf, "device error %d (inverted element?) at tet row %d", code, idx);
    status = set_error(ctx, code, buf);
  } else if (status == EBB_ERR_CG_BREAKDOWN) {
    char buf[128];
    snprintf(buf, sizeof buf, "PCG breakdown (p^T A p <= 0) at iteration %d", h.iter);
    set_error(ctx, status, buf);
  } else if (prm->fail_on_max_iters && h.iter >= prm->max_iters && rel > prm->rtol) {
    char buf[128];
    snprintf(buf, sizeof buf, "PCG not converged after %d iterations (rel residual %.3e)", h.iter, rel);
    status = set_error(ctx, EBB_ERR_NOT_CONVERGED, buf);
  }
  if (rep) rep->status = status;
  return status;
}

}  // namespace

ebb_status_t run_implicit_step(ebb_ctx_s* ctx, ebb_rel_s* tets, double* u, double* v, const void* pinned,
                               ebb_dtype_t pinned_dtype, const ebb_step_params_t* p, ebb_cg_report_t* rep) {
  if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, EBB_ERR_CUDA, "cudaSetDevice failed");
  if (tets->verts->size == 0) {
    if (rep) rep->status = EBB_OK;
    return EBB_OK;
  }
  ebb_status_t s = ensure_scratch(ctx, tets);
  if (s) return s;
  const bool f64 = p->precision == EBB_PREC_F64;
  if (tets->vperm) {
    // Reordered vertices: the step runs on the state in the internal order.
    StepScratch* sc = tets->step;
    const int nv = sc->nv;
    cudaError_t e = cudaSuccess;
    if (!sc->u_int) e = cudaMalloc(&sc->u_int, (size_t)3 * nv * sizeof(double));
    if (e == cudaSuccess && !sc->v_int) e = cudaMalloc(&sc->v_int, (size_t)3 * nv * sizeof(double));
    if (e == cudaSuccess && !sc->pin_int) e = cudaMalloc(&sc->pin_int, (size_t)nv);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(ctx, EBB_ERR_NOMEM, "device allocation for the reordered state failed");
    }
    e = gather_vertex_field<double>(nv, tets->vperm, u, sc->u_int, ctx->stream);
    if (e == cudaSuccess) e = gather_vertex_field<double>(nv, tets->vperm, v, sc->v_int, ctx->stream);
    if (e == cudaSuccess)
      e = pinned_dtype == EBB_I32
              ? gather_pinned<int>(nv, tets->vperm, (const int*)pinned, sc->pin_int, ctx->stream)
              : gather_pinned<unsigned char>(nv, tets->vperm, (const unsigned char*)pinned, sc->pin_int, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "reordering the state");
    const ebb_status_t r = f64 ? step_impl<double, unsigned char>(ctx, tets, sc->u_int, sc->v_int, sc->pin_int, p, rep)
                               : step_impl<float, unsigned char>(ctx, tets, sc->u_int, sc->v_int, sc->pin_int, p, rep);
    e = scatter_vertex_field(nv, tets->vperm, sc->u_int, u, ctx->stream);
    if (e == cudaSuccess) e = scatter_vertex_field(nv, tets->vperm, sc->v_int, v, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "restoring the state order");
    return r;
  }
  if (pinned_dtype == EBB_I32) {
    return f64 ? step_impl<double, int>(ctx, tets, u, v, (const int*)pinned, p, rep)
               : step_impl<float, int>(ctx, tets, u, v, (const int*)pinned, p, rep);
  }
  return f64 ? step_impl<double, unsigned char>(ctx, tets, u, v, (const unsigned char*)pinned, p, rep)
             : step_impl<float, unsigned char>(ctx, tets, u, v, (const unsigned char*)pinned, p, rep);
}

ebb_status_t run_step_vjp(ebb_ctx_s* ctx, ebb_rel_s* tets, const double* u, const double* v, const double* v_next,
                          const void* pinned, ebb_dtype_t pinned_dtype, double* gu, double* gv, double* gmu,
                          double* glam, const ebb_step_params_t* p, ebb_cg_report_t* rep) {
  if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, EBB_ERR_CUDA, "cudaSetDevice failed");
  if (tets->verts->size == 0) {
    if (rep) rep->status = EBB_OK;
    return EBB_OK;
  }
  ebb_status_t s = ensure_scratch(ctx, tets);
  if (s) return s;
  StepScratch* sc = tets->step;
  if (!sc->vjp_w) {
    const size_t n = (size_t)3 * sc->nv * sizeof(double);
    cudaError_t e = cudaMalloc(&sc->vjp_w, n);
    if (e == cudaSuccess) e = cudaMalloc(&sc->vjp_kl, n);
    if (e == cudaSuccess) e = cudaMalloc(&sc->vjp_xq, n);
    if (e != cudaSuccess) {
      cudaFree(sc->vjp_w);
      cudaFree(sc->vjp_kl);
      cudaFree(sc->vjp_xq);
      sc->vjp_w = sc->vjp_kl = sc->vjp_xq = nullptr;
      cudaGetLastError();
      return set_error(ctx, EBB_ERR_NOMEM, "device allocation for the step VJP failed");
    }
  }
  VjpArgs a{gu, gv, gmu, glam, v_next};
  // The forward solve reads u and v only; the finish step is replaced by the
  // adjoint, so neither is written.
  if (pinned_dtype == EBB_I32)
    return step_impl<double, int>(ctx, tets, const_cast<double*>(u), const_cast<double*>(v), (const int*)pinned, p,
                                  rep, &a);
  return step_impl<double, unsigned char>(ctx, tets, const_cast<double*>(u), const_cast<double*>(v),
                                          (const unsigned char*)pinned, p, rep, &a);
}

}  // namespace ebb
