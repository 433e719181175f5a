// Implicit step that allocates nothing: ebb_cg_implicit_step_noalloc.
//
// For callers that cannot allocate device memory.  The same linearised
// backward-Euler step and Jacobi-preconditioned CG as ebb_cg_implicit_step
// (FP64, atomic scatter), but every byte of working memory lives in one
// file-scope device array, carved into fixed regions for the largest
// supported mesh.  Host code cannot use the array's name as a device
// address, so the address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "ebb_internal.h"
#include "tet_math.cuh"

namespace ebb {
namespace noalloc {

constexpr int kMaxV = EBB_NOALLOC_MAX_VERTS;
constexpr int kMaxT = EBB_NOALLOC_MAX_TETS;
constexpr int kThreads = 256;
constexpr int kBlocks = 64;   // vector kernels: fixed grid, partial sums per block
constexpr int kChunk = 8;     // CG iterations between status reads (even)

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of the regions inside the scratch array.
constexpr size_t kOffB = 0;                                           // 9 planes of kMaxT
constexpr size_t kOffV = align256(kOffB + sizeof(double) * 9 * kMaxT);  // kMaxT
constexpr size_t kOffMass = align256(kOffV + sizeof(double) * kMaxT);   // kMaxV
constexpr size_t kVec = sizeof(double) * 3 * kMaxV;
constexpr size_t kOffF = align256(kOffMass + sizeof(double) * kMaxV);   // force
constexpr size_t kOffKv = align256(kOffF + kVec);                       // K v
constexpr size_t kOffD = align256(kOffKv + kVec);                       // diag K
constexpr size_t kOffKp = align256(kOffD + kVec);                       // K p
constexpr size_t kOffR = align256(kOffKp + kVec);
constexpr size_t kOffP = align256(kOffR + kVec);
constexpr size_t kOffY = align256(kOffP + kVec);
constexpr size_t kOffDinv = align256(kOffY + kVec);
constexpr size_t kOffPart = align256(kOffDinv + kVec);                  // 2 sets of kBlocks pairs
constexpr size_t kOffSc = align256(kOffPart + sizeof(double) * 4 * kBlocks);
constexpr size_t kOffErr = align256(kOffSc + 256);
constexpr size_t kBytes = align256(kOffErr + 4 * sizeof(int));

struct Scalars {
  double rz[2];
  double rr;
  double bb;
  int active[2];
  int iter;
  int status;
};
static_assert(sizeof(Scalars) <= 256, "scalar region");

}  // namespace noalloc
}  // namespace ebb

// The working memory of every ebb_cg_implicit_step_noalloc call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ebb::noalloc::kBytes];

namespace ebb {
namespace noalloc {
namespace {

struct Regions {
  double *B, *V, *mass, *f, *kv, *d, *kp, *r, *p, *y, *dinv, *part;
  Scalars* sc;
  int* err;
};

Regions carve(unsigned char* base) {
  Regions g;
  g.B = reinterpret_cast<double*>(base + kOffB);
  g.V = reinterpret_cast<double*>(base + kOffV);
  g.mass = reinterpret_cast<double*>(base + kOffMass);
  g.f = reinterpret_cast<double*>(base + kOffF);
  g.kv = reinterpret_cast<double*>(base + kOffKv);
  g.d = reinterpret_cast<double*>(base + kOffD);
  g.kp = reinterpret_cast<double*>(base + kOffKp);
  g.r = reinterpret_cast<double*>(base + kOffR);
  g.p = reinterpret_cast<double*>(base + kOffP);
  g.y = reinterpret_cast<double*>(base + kOffY);
  g.dinv = reinterpret_cast<double*>(base + kOffDinv);
  g.part = reinterpret_cast<double*>(base + kOffPart);
  g.sc = reinterpret_cast<Scalars*>(base + kOffSc);
  g.err = reinterpret_cast<int*>(base + kOffErr);
  return g;
}

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch names a host-side stand-in, so the address the kernels
// use is looked up on every call: the lookup allocates nothing, and a cached
// address would go stale if the module were reloaded (after a
// cudaDeviceReset, for instance).
cudaError_t scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

__device__ __forceinline__ void raise(int* err, int code, int idx) {
  if (atomicCAS(err, 0, code) == 0) err[1] = idx;
}

// Validate keys, form B = Dm^-1 and V = det(Dm)/6 (FP64), zero accumulators
// and the status word.
__global__ void setup_kernel(int nv, int nt, const int* __restrict__ keys, const double* __restrict__ X,
                             Regions g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * nv) {
    g.f[i] = 0.0;
    g.kv[i] = 0.0;
    g.d[i] = 0.0;
    g.kp[i] = 0.0;
  }
  if (i < nv) g.mass[i] = 0.0;
  if (i >= nt) return;
  int k[4];
  for (int a = 0; a < 4; ++a) {
    k[a] = keys[(size_t)a * nt + i];
    if (k[a] < 0 || k[a] >= nv) {
      raise(g.err, EBB_ERR_KEY, i);
      return;
    }
  }
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b)
      if (k[a] == k[b]) {
        raise(g.err, EBB_ERR_KEY, i);
        return;
      }
  double D[9];
  for (int c = 0; c < 3; ++c) {
    const double x0 = X[(size_t)c * nv + k[0]];
    for (int j = 0; j < 3; ++j) D[c * 3 + j] = X[(size_t)c * nv + k[j + 1]] - x0;
  }
  const double c00 = D[4] * D[8] - D[5] * D[7], c01 = D[5] * D[6] - D[3] * D[8], c02 = D[3] * D[7] - D[4] * D[6];
  const double det = D[0] * c00 + D[1] * c01 + D[2] * c02;
  if (!(det > 0.0)) {
    raise(g.err, EBB_ERR_INVERTED, i);
    return;
  }
  const double id = 1.0 / det;
  const double Bm[9] = {c00 * id,
                        (D[2] * D[7] - D[1] * D[8]) * id,
                        (D[1] * D[5] - D[2] * D[4]) * id,
                        c01 * id,
                        (D[0] * D[8] - D[2] * D[6]) * id,
                        (D[2] * D[3] - D[0] * D[5]) * id,
                        c02 * id,
                        (D[1] * D[6] - D[0] * D[7]) * id,
                        (D[0] * D[4] - D[1] * D[3]) * id};
  for (int q = 0; q < 9; ++q) g.B[(size_t)q * kMaxT + i] = Bm[q];
  g.V[i] = det / 6.0;
}

__global__ void mass_kernel(int nv, int nt, const int* __restrict__ keys, double rho, Regions g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double q = 0.25 * rho * g.V[t];
  for (int a = 0; a < 4; ++a) atomicAdd(g.mass + keys[(size_t)a * nt + t], q);
}

// One thread per tet: force, K w and diag K (FULL) or K w only, atomics.
template <int MODEL, bool FULL>
__global__ void element_kernel(int nv, int nt, const int* __restrict__ keys, double mu, double lam,
                               const double* __restrict__ u, const double* __restrict__ w, Regions g,
                               double* Kw_out, const int* active) {
  if (active != nullptr && *active == 0) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int k[4];
  for (int a = 0; a < 4; ++a) k[a] = keys[(size_t)a * nt + t];
  double B[9];
  for (int q = 0; q < 9; ++q) B[q] = g.B[(size_t)q * kMaxT + t];
  const double V = g.V[t];
  double Du[9], Dw[9], G[9], dF[9];
  for (int c = 0; c < 3; ++c) {
    const double u0 = u[(size_t)c * nv + k[0]], w0 = w[(size_t)c * nv + k[0]];
    for (int j = 0; j < 3; ++j) {
      Du[c * 3 + j] = u[(size_t)c * nv + k[j + 1]] - u0;
      Dw[c * 3 + j] = w[(size_t)c * nv + k[j + 1]] - w0;
    }
  }
  mm(Du, B, G);
  mm(Dw, B, dF);
  StvkState<double> sv;
  NhState<double> sn;
  double P[9], dP[9];
  if (MODEL == EBB_STVK) {
    stvk_state(G, mu, lam, sv);
    stvk_dP(sv, mu, lam, dF, dP);
    if (FULL) stvk_P(sv, P);
  } else {
    if (!nh_state(G, sn)) {
      raise(g.err, EBB_ERR_INVERTED, t);
      return;
    }
    nh_dP(sn, mu, lam, dF, dP);
    if (FULL) nh_P(sn, mu, lam, P);
  }
  for (int c = 0; c < 3; ++c) {
    double sf = 0.0, sk = 0.0;
    for (int a = 1; a <= 3; ++a) {
      const double* b = B + (a - 1) * 3;
      const double kv = V * (dP[c * 3] * b[0] + dP[c * 3 + 1] * b[1] + dP[c * 3 + 2] * b[2]);
      atomicAdd(Kw_out + (size_t)c * nv + k[a], kv);
      sk -= kv;
      if (FULL) {
        const double fv = -V * (P[c * 3] * b[0] + P[c * 3 + 1] * b[1] + P[c * 3 + 2] * b[2]);
        atomicAdd(g.f + (size_t)c * nv + k[a], fv);
        sf -= fv;
      }
    }
    atomicAdd(Kw_out + (size_t)c * nv + k[0], sk);
    if (FULL) atomicAdd(g.f + (size_t)c * nv + k[0], sf);
  }
  if (FULL) {
    for (int a = 0; a < 4; ++a) {
      double b[3];
      for (int j = 0; j < 3; ++j) b[j] = a == 0 ? -(B[j] + B[3 + j] + B[6 + j]) : B[(a - 1) * 3 + j];
      double dg[3];
      if (MODEL == EBB_STVK)
        stvk_diag(sv, mu, lam, b, dg);
      else
        nh_diag(sn, mu, lam, b, dg);
      for (int c = 0; c < 3; ++c) atomicAdd(g.d + (size_t)c * nv + k[a], V * dg[c]);
    }
  }
}

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Sum (a, b) over the block; result in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kThreads / 32], sb[kThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = warp_sum(l < kThreads / 32 ? sa[l] : 0.0);
    b = warp_sum(l < kThreads / 32 ? sb[l] : 0.0);
  }
  __syncthreads();
}

// Fixed-order sum of the per-block partials; every thread gets the result.
__device__ __forceinline__ void sum_partials(const double* part, double& a, double& b) {
  __shared__ double ra, rb;
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < kBlocks; i += kThreads) {
    x += part[2 * i];
    y += part[2 * i + 1];
  }
  block_sum2(x, y);
  if (threadIdx.x == 0) {
    ra = x;
    rb = y;
  }
  __syncthreads();
  a = ra;
  b = rb;
}

struct StepArgs {
  int nv;
  double dt, g0, g1, g2, rtol;
  int max_iters;
};

__device__ __forceinline__ bool pinned_at(const uint8_t* pin, int v) { return pin != nullptr && pin[v] != 0; }

__global__ void init_kernel(StepArgs c, const uint8_t* __restrict__ pin, Regions g) {
  const int n = 3 * c.nv;
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += kBlocks * kThreads) {
    const int comp = i / c.nv, vtx = i - comp * c.nv;
    double b = 0.0, di = 1.0;
    if (!pinned_at(pin, vtx)) {
      const double m = g.mass[vtx];
      const double gc = comp == 0 ? c.g0 : (comp == 1 ? c.g1 : c.g2);
      b = c.dt * (g.f[i] + m * gc - c.dt * g.kv[i]);
      di = 1.0 / (m + c.dt * c.dt * g.d[i]);
    }
    const double z = b * di;
    g.r[i] = b;
    g.p[i] = z;
    g.y[i] = 0.0;
    g.dinv[i] = di;
    rz += b * z;
    rr += b * b;
  }
  block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    g.part[2 * blockIdx.x] = rz;
    g.part[2 * blockIdx.x + 1] = rr;
  }
}

__global__ void start_kernel(StepArgs c, Regions g) {
  double rz, rr;
  sum_partials(g.part, rz, rr);
  if (threadIdx.x == 0) {
    g.sc->rz[0] = rz;
    g.sc->rz[1] = 0.0;
    g.sc->rr = rr;
    g.sc->bb = rr;
    g.sc->iter = 0;
    g.sc->status = EBB_OK;
    g.sc->active[0] = (c.max_iters > 0 && sqrt(rr) > c.rtol * sqrt(rr)) ? 1 : 0;
    g.sc->active[1] = 0;
  }
}

__global__ void pq_kernel(StepArgs c, int s, const uint8_t* __restrict__ pin, Regions g) {
  if (!g.sc->active[s]) return;
  const int n = 3 * c.nv;
  double pq = 0.0, zero = 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += kBlocks * kThreads) {
    const int vtx = i % c.nv;
    if (pinned_at(pin, vtx)) continue;
    const double pi = g.p[i];
    pq += pi * (g.mass[vtx] * pi + c.dt * c.dt * g.kp[i]);
  }
  block_sum2(pq, zero);
  if (threadIdx.x == 0) {
    g.part[2 * blockIdx.x] = pq;
    g.part[2 * blockIdx.x + 1] = 0.0;
  }
}

__global__ void update_kernel(StepArgs c, int s, const uint8_t* __restrict__ pin, Regions g) {
  if (!g.sc->active[s]) return;
  double pq, unused;
  sum_partials(g.part, pq, unused);
  if (!(pq > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) g.sc->status = EBB_ERR_CG_BREAKDOWN;
    return;
  }
  const double alpha = g.sc->rz[s] / pq;
  const int n = 3 * c.nv;
  double rz = 0.0, rr = 0.0;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += kBlocks * kThreads) {
    const int vtx = i % c.nv;
    if (pinned_at(pin, vtx)) continue;
    const double pi = g.p[i];
    const double q = g.mass[vtx] * pi + c.dt * c.dt * g.kp[i];
    g.y[i] += alpha * pi;
    const double ri = g.r[i] - alpha * q;
    g.r[i] = ri;
    rz += ri * (ri * g.dinv[i]);
    rr += ri * ri;
  }
  block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    g.part[2 * kBlocks + 2 * blockIdx.x] = rz;
    g.part[2 * kBlocks + 2 * blockIdx.x + 1] = rr;
  }
}

__global__ void pupdate_kernel(StepArgs c, int s, Regions g) {
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  if (!g.sc->active[s] || g.sc->status != EBB_OK) {
    if (lead) g.sc->active[s ^ 1] = 0;
    return;
  }
  double rz_new, rr;
  sum_partials(g.part + 2 * kBlocks, rz_new, rr);
  const double beta = rz_new / g.sc->rz[s];
  const int n = 3 * c.nv;
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += kBlocks * kThreads) {
    g.p[i] = g.r[i] * g.dinv[i] + beta * g.p[i];
    g.kp[i] = 0.0;
  }
  if (lead) {
    const int it = g.sc->iter + 1;
    g.sc->iter = it;
    g.sc->rz[s ^ 1] = rz_new;
    g.sc->rr = rr;
    g.sc->active[s ^ 1] = (it < c.max_iters && sqrt(rr) > c.rtol * sqrt(g.sc->bb)) ? 1 : 0;
  }
}

__global__ void finish_kernel(int n, double dt, Regions g, double* u, double* v) {
  for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += kBlocks * kThreads) {
    const double vi = v[i] + g.y[i];
    v[i] = vi;
    u[i] += dt * vi;
  }
}

template <int MODEL>
cudaError_t launch_elements(bool full, int nv, int nt, const int* keys, double mu, double lam, const double* u,
                            const double* w, const Regions& g, double* out, const int* active, cudaStream_t st) {
  const int grid = (nt + kThreads - 1) / kThreads;
  if (grid == 0) return cudaSuccess;
  if (full)
    element_kernel<MODEL, true><<<grid, kThreads, 0, st>>>(nv, nt, keys, mu, lam, u, w, g, out, active);
  else
    element_kernel<MODEL, false><<<grid, kThreads, 0, st>>>(nv, nt, keys, mu, lam, u, w, g, out, active);
  return cudaGetLastError();
}

ebb_status_t run(cudaStream_t st, int nv, int nt, const int* keys, const double* X, double* u, double* v,
                 const uint8_t* pin, const ebb_step_params_t* prm, ebb_cg_report_t* rep) {
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return EBB_ERR_CUDA;
  const Regions g = carve(base);
  const int n = 3 * nv;
  cudaError_t e = cudaMemsetAsync(g.err, 0, 4 * sizeof(int), st);
  if (e != cudaSuccess) return EBB_ERR_CUDA;
  const int sgrid = ((nt > n ? nt : n) + kThreads - 1) / kThreads;
  setup_kernel<<<sgrid, kThreads, 0, st>>>(nv, nt, keys, X, g);
  // Keys are read back as valid before any kernel indexes through them.
  int herr[4] = {0, 0, 0, 0};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(herr, g.err, sizeof herr, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return EBB_ERR_CUDA;
  if (herr[0] != 0) return herr[0];
  if (nt > 0) mass_kernel<<<(nt + kThreads - 1) / kThreads, kThreads, 0, st>>>(nv, nt, keys, prm->rho, g);

  StepArgs c;
  memset(&c, 0, sizeof c);
  c.nv = nv;
  c.dt = prm->dt;
  c.g0 = prm->gravity[0];
  c.g1 = prm->gravity[1];
  c.g2 = prm->gravity[2];
  c.rtol = prm->rtol;
  c.max_iters = prm->max_iters;
  const bool stvk = prm->model == EBB_STVK;
  e = stvk ? launch_elements<EBB_STVK>(true, nv, nt, keys, prm->mu, prm->lambda, u, v, g, g.kv, nullptr, st)
           : launch_elements<EBB_NEOHOOKEAN>(true, nv, nt, keys, prm->mu, prm->lambda, u, v, g, g.kv, nullptr, st);
  if (e != cudaSuccess) return EBB_ERR_CUDA;
  init_kernel<<<kBlocks, kThreads, 0, st>>>(c, pin, g);
  start_kernel<<<1, kThreads, 0, st>>>(c, g);
  if (cudaGetLastError() != cudaSuccess) return EBB_ERR_CUDA;

  Scalars h;
  ebb_status_t status = EBB_OK;
  int launched = 0;
  while (true) {
    for (int k = 0; k < kChunk; ++k) {
      const int par = k & 1;
      e = stvk ? launch_elements<EBB_STVK>(false, nv, nt, keys, prm->mu, prm->lambda, u, g.p, g, g.kp,
                                           &g.sc->active[par], st)
               : launch_elements<EBB_NEOHOOKEAN>(false, nv, nt, keys, prm->mu, prm->lambda, u, g.p, g, g.kp,
                                                 &g.sc->active[par], st);
      if (e != cudaSuccess) return EBB_ERR_CUDA;
      pq_kernel<<<kBlocks, kThreads, 0, st>>>(c, par, pin, g);
      update_kernel<<<kBlocks, kThreads, 0, st>>>(c, par, pin, g);
      pupdate_kernel<<<kBlocks, kThreads, 0, st>>>(c, par, g);
    }
    launched += kChunk;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, g.sc, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return EBB_ERR_CUDA;
    if (h.status != EBB_OK) {
      status = h.status;
      break;
    }
    if (!h.active[h.iter & 1] || h.iter >= prm->max_iters) break;
    if (launched > prm->max_iters + 2 * kChunk) break;
  }
  finish_kernel<<<kBlocks, kThreads, 0, st>>>(n, prm->dt, g, u, v);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, g.sc, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(herr, g.err, sizeof herr, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return EBB_ERR_CUDA;
  const double rel = h.bb > 0.0 ? std::sqrt(h.rr / h.bb) : 0.0;
  if (rep) {
    rep->iters = h.iter;
    rep->rel_residual = rel;
  }
  if (herr[0] != 0)
    status = herr[0];
  else if (status == EBB_OK && prm->fail_on_max_iters && h.iter >= prm->max_iters && rel > prm->rtol)
    status = EBB_ERR_NOT_CONVERGED;
  return status;
}

}  // namespace
}  // namespace noalloc
}  // namespace ebb

extern "C" ebb_status_t ebb_cg_implicit_step_noalloc(void* cuda_stream, int32_t n_verts, int32_t n_tets,
                                                     const int32_t* keys, const double* X, double* u, double* v,
                                                     const uint8_t* pinned, const ebb_step_params_t* params,
                                                     ebb_cg_report_t* report) {
  if (report) {
    report->iters = 0;
    report->rel_residual = 0.0;
    report->status = EBB_ERR_ARG;
  }
  if (!params || n_verts < 0 || n_tets < 0 || n_verts > EBB_NOALLOC_MAX_VERTS || n_tets > EBB_NOALLOC_MAX_TETS)
    return EBB_ERR_ARG;
  if (params->precision != EBB_PREC_F64 || (params->model != EBB_STVK && params->model != EBB_NEOHOOKEAN) ||
      params->flags != 0)
    return EBB_ERR_ARG;
  if (!(params->dt > 0.0) || !(params->rho > 0.0) || params->max_iters < 0 || !(params->rtol >= 0.0))
    return EBB_ERR_ARG;
  if (n_verts > 0 && (!X || !u || !v)) return EBB_ERR_ARG;
  if (n_tets > 0 && !keys) return EBB_ERR_ARG;
  if (n_verts == 0) {
    if (n_tets > 0) return EBB_ERR_KEY;
    if (report) report->status = EBB_OK;
    return EBB_OK;
  }
  const ebb_status_t s = ebb::noalloc::run((cudaStream_t)cuda_stream, n_verts, n_tets, keys, X, u, v, pinned,
                                           params, report);
  if (report) report->status = s;
  return s;
}
