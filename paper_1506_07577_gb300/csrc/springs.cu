// Spring-mass system on the edge relation: the paper's introductory example
// (Section 4.1, Figure 1) as a second workload on the same runtime.
//
// The springs are the mesh's edges (the edge relation of EBB_FINALIZE_EDGES,
// each vertex's row listing its neighbours).  Per step, one kernel walks
// every vertex's row -- computeInternalForces, a per-vertex loop over the
// directed edges leaving it, one thread per vertex summing its springs in row
// order (no atomics; bitwise reproducible; measured faster than 2, 4 or 8
// lanes per vertex with a shuffle tree) -- and then applies the force to that
// vertex (applyForces):
//   f_v = sum_h K (L_vh dir - dq),  dq = q_v - q_h,  dir = dq / |dq|
//   qdd = f_v / m_v,  q_v += qd_v dt + qdd dt^2 / 2,  qd_v += qdd dt
// (the restoring reading of the figure's force; a zero-length dq gives no
// direction and a vertex with m <= 0 does not move).  Positions are read from
// one buffer and written to another (the two kernels of the figure, whose
// phases keep force accumulation and position update apart, fused by double
// buffering), velocities in place.  measureTotalEnergy is a two-pass sum of
// m |qd|^2 / 2 in FP64 in a fixed order.
#include <algorithm>

#include "ebb_internal.h"

namespace ebb {

namespace {

constexpr int kSpringThreads = 256;
constexpr int kEnergyBlocks = 304;

// 1 / |dq| from |dq|^2 (CUDA's reciprocal square roots: within 2 ulp in
// FP32 and 1 ulp in FP64, one call where a square root and a division
// would be two; FP64 division and square root are long sequences on GB300's
// FP64 pipe).
template <typename T>
__device__ __forceinline__ T inv_len(T n2);
template <>
__device__ __forceinline__ float inv_len<float>(float n2) { return rsqrtf(n2); }
template <>
__device__ __forceinline__ double inv_len<double>(double n2) { return rsqrt(n2); }

template <typename T>
__global__ void __launch_bounds__(kSpringThreads)
rest_length_kernel(int nv, const int* __restrict__ row_off, const int* __restrict__ col, const T* __restrict__ X,
                   T* rest) {
  const int r = blockIdx.x * kSpringThreads + threadIdx.x;
  if (r >= nv) return;
  for (int k = row_off[r]; k < row_off[r + 1]; ++k) {
    const int h = col[k];
    T s = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T d = X[(size_t)c * nv + h] - X[(size_t)c * nv + r];
      s += d * d;
    }
    rest[k] = sqrt(s);
  }
}

template <typename T>
__global__ void __launch_bounds__(kSpringThreads)
spring_step_kernel(int nv, const int* __restrict__ row_off, const int* __restrict__ col, const T* __restrict__ rest,
                   const T* __restrict__ mass, T k, T dt, const T* __restrict__ qin, T* __restrict__ qout, T* qd) {
  const int r = blockIdx.x * kSpringThreads + threadIdx.x;
  if (r >= nv) return;
  T f[3] = {T(0), T(0), T(0)};
  T qr[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) qr[c] = qin[(size_t)c * nv + r];
  const int k1 = row_off[r + 1];
  for (int e = row_off[r]; e < k1; ++e) {
    const int h = col[e];
    if (h == r) continue;   // the self-loop of the edge relation
    T dq[3], n2 = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dq[c] = qr[c] - qin[(size_t)c * nv + h];
      n2 += dq[c] * dq[c];
    }
    const T s = n2 > T(0) ? rest[e] * inv_len(n2) : T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] += k * (s * dq[c] - dq[c]);
  }
  const T m = mass[r];
  const T im = m > T(0) ? T(1) / m : T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const size_t i = (size_t)c * nv + r;
    const T a = f[c] * im;
    const T v = qd[i];
    qout[i] = qr[c] + v * dt + T(0.5) * a * dt * dt;
    qd[i] = v + a * dt;
  }
}

// Per-block partial sums of m |qd|^2 / 2 (FP64), block order fixed.
template <typename T>
__global__ void __launch_bounds__(kSpringThreads)
energy_partial_kernel(int nv, const T* __restrict__ qd, const T* __restrict__ mass, double* part) {
  __shared__ double s[kSpringThreads];
  double e = 0.0;
  for (int v = blockIdx.x * kSpringThreads + threadIdx.x; v < nv; v += gridDim.x * kSpringThreads) {
    double q2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double x = (double)qd[(size_t)c * nv + v];
      q2 += x * x;
    }
    e += 0.5 * (double)mass[v] * q2;
  }
  s[threadIdx.x] = e;
  __syncthreads();
  for (int w = kSpringThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ a, B* __restrict__ b, int n) {
  const int i = blockIdx.x * kSpringThreads + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

template <typename A, typename B>
cudaError_t convert_array(const A* a, B* b, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  convert_kernel<A, B><<<(n + kSpringThreads - 1) / kSpringThreads, kSpringThreads, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

__global__ void energy_final_kernel(const double* part, int n, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double e = 0.0;
  for (int i = 0; i < n; ++i) e += part[i];
  *out = e;
}

template <typename T>
cudaError_t springs_run_t(ebb_rel_s* tets, T* q, T* qd, const T* mass, double k, double dt, int steps, double* energy,
                          cudaStream_t st) {
  EdgeIndex& E = tets->edges;
  const int p = sizeof(T) == 4 ? 0 : 1;
  const int nv = (int)tets->verts->size;
  if (E.qbuf[p] == nullptr) {
    cudaError_t e = cudaMalloc(&E.qbuf[p], std::max<size_t>(1, (size_t)3 * nv) * sizeof(T));
    if (e != cudaSuccess) {
      E.qbuf[p] = nullptr;
      return e;
    }
  }
  T* bufs[2] = {q, static_cast<T*>(E.qbuf[p])};
  const T* rest = static_cast<const T*>(E.rest[p]);
  const int grid = (nv + kSpringThreads - 1) / kSpringThreads;
  for (int s = 0; s < steps && nv > 0; ++s) {
    spring_step_kernel<T><<<grid, kSpringThreads, 0, st>>>(nv, E.row_off, E.col, rest, mass, (T)k, (T)dt,
                                                           bufs[s & 1], bufs[(s + 1) & 1], qd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if ((steps & 1) && nv > 0) {
    cudaError_t e = cudaMemcpyAsync(q, bufs[1], (size_t)3 * nv * sizeof(T), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  if (energy != nullptr) {
    double* dpart = E.epart;
    energy_partial_kernel<T><<<kEnergyBlocks, kSpringThreads, 0, st>>>(nv, qd, mass, dpart);
    energy_final_kernel<<<1, 32, 0, st>>>(dpart, kEnergyBlocks, dpart + kEnergyBlocks);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(energy, dpart + kEnergyBlocks, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t springs_init(ebb_rel_s* tets, const void* X, bool f64, cudaStream_t st) {
  EdgeIndex& E = tets->edges;
  const int nv = (int)tets->verts->size;
  const size_t n = std::max<size_t>(1, (size_t)E.nnzb);
  for (int p = 0; p < 2; ++p)
    if (E.rest[p] == nullptr) {
      cudaError_t e = cudaMalloc(&E.rest[p], n * (p == 0 ? sizeof(float) : sizeof(double)));
      if (e != cudaSuccess) {
        E.rest[p] = nullptr;
        return e;
      }
    }
  if (E.epart == nullptr) {
    cudaError_t e = cudaMalloc(&E.epart, (kEnergyBlocks + 1) * sizeof(double));
    if (e != cudaSuccess) {
      E.epart = nullptr;
      return e;
    }
  }
  if (nv == 0) {
    E.springs_ready = true;
    return cudaSuccess;
  }
  const int grid = (nv + kSpringThreads - 1) / kSpringThreads;
  // Lengths in the positions' precision, then the other precision's copy.
  if (f64) {
    rest_length_kernel<double><<<grid, kSpringThreads, 0, st>>>(nv, E.row_off, E.col, (const double*)X,
                                                                (double*)E.rest[1]);
  } else {
    rest_length_kernel<float><<<grid, kSpringThreads, 0, st>>>(nv, E.row_off, E.col, (const float*)X,
                                                               (float*)E.rest[0]);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = f64 ? convert_array((const double*)E.rest[1], (float*)E.rest[0], E.nnzb, st)
          : convert_array((const float*)E.rest[0], (double*)E.rest[1], E.nnzb, st);
  if (e == cudaSuccess) E.springs_ready = true;
  return e;
}

cudaError_t springs_run(ebb_rel_s* tets, void* q, void* qd, const void* mass, bool f64, double k, double dt, int steps,
                        double* energy, cudaStream_t st) {
  return f64 ? springs_run_t<double>(tets, (double*)q, (double*)qd, (const double*)mass, k, dt, steps, energy, st)
             : springs_run_t<float>(tets, (float*)q, (float*)qd, (const float*)mass, k, dt, steps, energy, st);
}

}  // namespace ebb
