// Batched implicit step: many independent meshes, one launch per kernel.
//
// The meshes are concatenated in one verts/tets relation pair; the I32
// vertex field named by `batch` gives each vertex its mesh id, with the
// vertices of a mesh contiguous and ids increasing along the relation (and
// finalize, seeing verts.batch, keeps each mesh's tets together and rejects
// tets that join two meshes).  Every element map runs once over all meshes'
// tiles (the persistent tiled map: one launch covers the whole batch); the
// CG state is per mesh.  The vector kernels use a block table: each block
// covers up to kBT vertices of one mesh, so a mesh's dot products are the
// fixed-order sum of its own blocks' partials (deterministic), finished by
// the mesh's last block to arrive, which also advances that mesh's scalars.
// A mesh whose solve has ended stops updating; the element map is skipped
// entirely once no mesh is active.  The same step as Section 7.2 / 7.3 per
// mesh: A = M + dt^2 K, b = dt (f + M g - dt K v), Jacobi PCG, v += dv,
// u += dt v.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "ebb_internal.h"

namespace ebb {
namespace {

constexpr int kBT = 256;     // threads (vertices) per block
constexpr int kChunk = 8;    // CG iterations per captured graph (even)

struct MeshCg {
  double rz[2];
  double rr, bb, alpha, beta;
  int active[2];
  int iter;
  int status;
  unsigned count[3];
  unsigned pad;
};

struct BatchTable {
  int nblocks;
  const int* blk_mesh;   // mesh of block b
  const int* blk_v0;     // first vertex of block b
  const int* blk_v1;     // one past its last vertex
  const int* mesh_blk0;  // first block of mesh m
  const int* mesh_nblk;  // blocks of mesh m
};

struct BatchConst {
  int nv;
  double dt;
  double g[3];
  double rtol;
  int max_iters;
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Block sum of (a, b), fixed order, result in thread 0.  FP64 adds are slow
// on GB300, so values go through shared memory and one warp adds them
// (kBT/32 per lane, then a shuffle tree) instead of a shuffle tree per warp.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kBT], sb[kBT];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = 0.0, y = 0.0;
#pragma unroll
    for (int i = 0; i < kBT / 32; ++i) {
      x += sa[threadIdx.x + 32 * i];
      y += sb[threadIdx.x + 32 * i];
    }
    a = warp_sum(x);
    b = warp_sum(y);
  }
  __syncthreads();
}

// dt^2 times a K p entry in FP64 (in FP32 first when K p is FP32).
__device__ __forceinline__ double dt2_times(float kp, double dt2) { return (double)((float)dt2 * kp); }
__device__ __forceinline__ double dt2_times(double kp, double dt2) { return dt2 * kp; }

// Per-mesh two-pass sum: block partial to part[2*b]; the mesh's last block
// sums its blocks' partials in block order and returns true with the totals.
__device__ __forceinline__ bool mesh_reduce_last(double& a, double& b, double* part, unsigned* counter, int blk0,
                                                 int nblk) {
  __shared__ unsigned s_last;
  __shared__ double ra, rb;
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
    __threadfence();
    s_last = atomicAdd(counter, 1u) == (unsigned)nblk - 1u ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kBT) {
    x += __ldcg(part + 2 * (blk0 + i));
    y += __ldcg(part + 2 * (blk0 + i) + 1);
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

__device__ __forceinline__ bool pinned_at(const unsigned char* pin, int v) { return pin != nullptr && pin[v] != 0; }

// Element-precision arrays of the step (f, K v, diag, K p accumulators and
// the FP32 copies of u and p) are vertex-interleaved in FP32 (AOS: 4 values
// per vertex), 3 planes otherwise; the FP64 CG vectors are always planes.
template <bool AOS>
__device__ __forceinline__ size_t eidx(int nv, int v, int comp) {
  return AOS ? 4 * (size_t)v + comp : (size_t)comp * nv + v;
}

template <typename T, bool AOS>
__global__ void __launch_bounds__(kBT)
batch_init_kernel(BatchConst c, BatchTable tb, const unsigned char* __restrict__ pin, const double* __restrict__ mass,
                  const T* __restrict__ acc_f, const T* __restrict__ acc_kv, const T* __restrict__ acc_d, double* r,
                  double* p, double* y, double* dinv, T* pe, double* part, MeshCg* sc, int* n_active) {
  const int m = tb.blk_mesh[blockIdx.x];
  const int v = tb.blk_v0[blockIdx.x] + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (v < tb.blk_v1[blockIdx.x]) {
    const bool pinned = pinned_at(pin, v);
    const double mv = mass[v];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const int i = comp * c.nv + v;
      const size_t ie = eidx<AOS>(c.nv, v, comp);
      double b = 0.0, di = 1.0;
      if (!pinned) {
        b = c.dt * ((double)acc_f[ie] + mv * c.g[comp] - c.dt * (double)acc_kv[ie]);
        di = 1.0 / (mv + c.dt * c.dt * (double)acc_d[ie]);
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
  }
  MeshCg& s = sc[m];
  if (mesh_reduce_last(rz, rr, part, &s.count[0], tb.mesh_blk0[m], tb.mesh_nblk[m]) && threadIdx.x == 0) {
    s.rz[0] = rz;
    s.rz[1] = 0.0;
    s.rr = rr;
    s.bb = rr;
    s.alpha = s.beta = 0.0;
    s.iter = 0;
    s.status = EBB_OK;
    const int act = (c.max_iters > 0 && sqrt(rr) > c.rtol * sqrt(rr)) ? 1 : 0;
    s.active[0] = act;
    s.active[1] = 0;
    if (act) atomicAdd(n_active, 1);
  }
}

template <typename T, bool AOS>
__global__ void __launch_bounds__(kBT)
batch_pq_kernel(BatchConst c, BatchTable tb, int s, const unsigned char* __restrict__ pin,
                const double* __restrict__ mass, const double* __restrict__ p, const T* __restrict__ acc_kp,
                double* __restrict__ qz, double* part, MeshCg* sc, int* n_active) {
  const int m = tb.blk_mesh[blockIdx.x];
  MeshCg& st = sc[m];
  if (!st.active[s]) return;
  const int v = tb.blk_v0[blockIdx.x] + threadIdx.x;
  const double dt2 = c.dt * c.dt;
  double pq = 0.0, zero = 0.0;
  if (v < tb.blk_v1[blockIdx.x] && !pinned_at(pin, v)) {
    const double mv = mass[v];
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const int i = comp * c.nv + v;
      const double pi = p[i];
      const double q = fma(mv, pi, dt2_times(acc_kp[eidx<AOS>(c.nv, v, comp)], dt2));
      qz[i] = q;
      pq = fma(pi, q, pq);
    }
  }
  if (mesh_reduce_last(pq, zero, part, &st.count[1], tb.mesh_blk0[m], tb.mesh_nblk[m]) && threadIdx.x == 0) {
    if (pq > 0.0) {
      st.alpha = st.rz[s] / pq;
    } else {
      st.alpha = 0.0;
      st.status = EBB_ERR_CG_BREAKDOWN;
      atomicSub(n_active, 1);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBT)
batch_update_kernel(BatchConst c, BatchTable tb, int s, const unsigned char* __restrict__ pin,
                    const double* __restrict__ p, const double* __restrict__ dinv, double* __restrict__ r,
                    double* __restrict__ y, double* __restrict__ qz, double* part, MeshCg* sc, int* n_active) {
  const int m = tb.blk_mesh[blockIdx.x];
  MeshCg& st = sc[m];
  if (!st.active[s] || st.status != EBB_OK) return;
  const double alpha = st.alpha;
  const int v = tb.blk_v0[blockIdx.x] + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (v < tb.blk_v1[blockIdx.x] && !pinned_at(pin, v)) {
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const int i = comp * c.nv + v;
      const double pi = p[i];
      y[i] = fma(alpha, pi, y[i]);
      const double ri = fma(-alpha, qz[i], r[i]);
      const double zi = ri * dinv[i];
      r[i] = ri;
      qz[i] = zi;
      rz = fma(ri, zi, rz);
      rr = fma(ri, ri, rr);
    }
  }
  if (mesh_reduce_last(rz, rr, part, &st.count[2], tb.mesh_blk0[m], tb.mesh_nblk[m]) && threadIdx.x == 0) {
    const int it = st.iter + 1;
    st.iter = it;
    st.beta = rz / st.rz[s];
    st.rz[s ^ 1] = rz;
    st.rr = rr;
    const int next = (it < c.max_iters && sqrt(rr) > c.rtol * sqrt(st.bb)) ? 1 : 0;
    st.active[s ^ 1] = next;
    if (!next) atomicSub(n_active, 1);
  }
}

template <typename T, bool AOS>
__global__ void __launch_bounds__(kBT)
batch_pupdate_kernel(BatchConst c, BatchTable tb, int s, const unsigned char* __restrict__ pin,
                     const double* __restrict__ qz, double* __restrict__ p, T* __restrict__ pe,
                     T* __restrict__ acc_kp, MeshCg* sc) {
  const int m = tb.blk_mesh[blockIdx.x];
  MeshCg& st = sc[m];
  if (!st.active[s] || st.status != EBB_OK) {
    if (threadIdx.x == 0 && blockIdx.x == tb.mesh_blk0[m]) st.active[s ^ 1] = 0;
    return;
  }
  const double beta = st.beta;
  const int v = tb.blk_v0[blockIdx.x] + threadIdx.x;
  if (v < tb.blk_v1[blockIdx.x]) {
    const bool pinned = pinned_at(pin, v);   // r = p = 0 there; z was not formed
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      const int i = comp * c.nv + v;
      const double pi = pinned ? 0.0 : fma(beta, p[i], qz[i]);
      const size_t ie = eidx<AOS>(c.nv, v, comp);
      p[i] = pi;
      if (pe) pe[ie] = (T)pi;
      acc_kp[ie] = T(0);
    }
  }
}

template <typename T, bool AOS>
__global__ void batch_prep_kernel(int nv, const double* __restrict__ u, const double* __restrict__ v, T* ue, T* ve,
                                  T* acc_f, T* acc_kv, T* acc_d, T* acc_kp, bool copy) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nv; x += gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < (AOS ? 4 : 3); ++k) {
      const size_t i = eidx<AOS>(nv, x, k);
      if (copy) {
        ue[i] = k < 3 ? (T)u[(size_t)k * nv + x] : T(0);
        ve[i] = k < 3 ? (T)v[(size_t)k * nv + x] : T(0);
      }
      acc_f[i] = acc_kv[i] = acc_d[i] = acc_kp[i] = T(0);
    }
  }
}

__global__ void batch_mass_kernel(int nv, const int* __restrict__ off, const int* __restrict__ ent,
                                  const double* __restrict__ V, double rho, double* mass) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int e = off[v]; e < off[v + 1]; ++e) s += V[ent[e] >> 2];
  mass[v] = 0.25 * rho * s;
}

__global__ void batch_finish_kernel(int n, double dt, const double* __restrict__ y, double* u, double* v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double vi = v[i] + y[i];
    v[i] = vi;
    u[i] += dt * vi;
  }
}

}  // namespace

// Scratch of the batched step (owned by the relation).
struct BatchScratch {
  int nv = 0, nmesh = 0;
  const void* batch_ptr = nullptr;
  int* table = nullptr;              // blk_mesh | blk_v0 | blk_v1 | mesh_blk0 | mesh_nblk
  BatchTable tb{};
  void* acc[4] = {nullptr, nullptr, nullptr, nullptr};
  void *ue = nullptr, *pe = nullptr;
  double *r = nullptr, *p = nullptr, *y = nullptr, *dinv = nullptr, *mass = nullptr, *part = nullptr;
  double* qz = nullptr;              // A p, then z = r / diag A, within one CG iteration
  MeshCg* sc = nullptr;
  int* n_active = nullptr;
  std::vector<MeshCg> h_sc;
  double rho = -1.0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t chunk = nullptr;
  std::vector<unsigned char> key;
};

void free_batch_scratch(ebb_rel_s* rel) {
  BatchScratch* s = rel->batch;
  if (!s) return;
  cudaFree(s->table);
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
  cudaFree(s->n_active);
  if (s->chunk) cudaGraphExecDestroy(s->chunk);
  if (s->ev) cudaEventDestroy(s->ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  rel->batch = nullptr;
}

namespace {

// Validate the batch field (ids non-decreasing from 0, each mesh non-empty)
// and build the block table.
ebb_status_t prepare_batch(ebb_ctx_s* ctx, ebb_rel_s* tets, const int* batch, int nmesh) {
  const int nv = (int)tets->verts->size;
  BatchScratch* s = tets->batch;
  if (s && s->nv == nv && s->nmesh == nmesh && s->batch_ptr == batch) return EBB_OK;
  free_batch_scratch(tets);
  std::vector<int> hb(nv);
  cudaError_t e = cudaMemcpyAsync(hb.data(), batch, sizeof(int) * nv, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "reading batch ids");
  std::vector<int> vstart(nmesh + 1, -1);
  int prev = -1;
  for (int v = 0; v < nv; ++v) {
    const int b = hb[v];
    if (b < 0 || b >= nmesh || b < prev)
      return set_error(ctx, EBB_ERR_ARG, "batch ids must be in [0, nbatch) and non-decreasing along verts");
    if (b != prev) {
      for (int q = prev + 1; q <= b; ++q) vstart[q] = v;
      prev = b;
    }
  }
  for (int q = prev + 1; q <= nmesh; ++q) vstart[q] = nv;
  std::vector<int> blk_mesh, blk_v0, blk_v1, mesh_blk0(nmesh), mesh_nblk(nmesh);
  for (int m = 0; m < nmesh; ++m) {
    mesh_blk0[m] = (int)blk_mesh.size();
    const int a = vstart[m], b = vstart[m + 1];
    if (b <= a) return set_error(ctx, EBB_ERR_ARG, "every batch id in [0, nbatch) needs at least one vertex");
    for (int v0 = a; v0 < b; v0 += kBT) {
      blk_mesh.push_back(m);
      blk_v0.push_back(v0);
      blk_v1.push_back(v0 + kBT < b ? v0 + kBT : b);
    }
    mesh_nblk[m] = (int)blk_mesh.size() - mesh_blk0[m];
  }
  const int nb = (int)blk_mesh.size();
  s = new BatchScratch();
  tets->batch = s;
  s->nv = nv;
  s->nmesh = nmesh;
  s->batch_ptr = batch;
  const size_t n = (size_t)3 * nv;
  e = cudaMalloc(&s->table, sizeof(int) * (3 * (size_t)nb + 2 * (size_t)nmesh));
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMalloc(&s->acc[i], n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->ue, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->pe, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->r, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->p, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->y, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->dinv, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->qz, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->mass, (size_t)nv * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->part, 2 * (size_t)nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->sc, (size_t)nmesh * sizeof(MeshCg));
  if (e == cudaSuccess) e = cudaMalloc(&s->n_active, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_batch_scratch(tets);
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, "device allocation for the batched step failed");
  }
  std::vector<int> host;
  host.insert(host.end(), blk_mesh.begin(), blk_mesh.end());
  host.insert(host.end(), blk_v0.begin(), blk_v0.end());
  host.insert(host.end(), blk_v1.begin(), blk_v1.end());
  host.insert(host.end(), mesh_blk0.begin(), mesh_blk0.end());
  host.insert(host.end(), mesh_nblk.begin(), mesh_nblk.end());
  e = cudaMemcpy(s->table, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_batch_scratch(tets);
    return cuda_check(ctx, e, "uploading the batch table");
  }
  s->tb.nblocks = nb;
  s->tb.blk_mesh = s->table;
  s->tb.blk_v0 = s->table + nb;
  s->tb.blk_v1 = s->table + 2 * nb;
  s->tb.mesh_blk0 = s->table + 3 * nb;
  s->tb.mesh_nblk = s->table + 3 * nb + nmesh;
  s->h_sc.resize(nmesh);
  return EBB_OK;
}

template <typename T>
ebb_status_t batch_impl(ebb_ctx_s* ctx, ebb_rel_s* tets, double* u, double* v, const unsigned char* pin,
                        const ebb_step_params_t* prm, int nmesh, ebb_cg_report_t* reps) {
  const bool mixed = sizeof(T) == 4;
  BatchScratch* s = tets->batch;
  const int nv = s->nv;
  const int n = 3 * nv;
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
  if (s->rho != prm->rho) {
    batch_mass_kernel<<<(nv + 255) / 256, 256, 0, st>>>(nv, tets->vindex.off, tets->vindex.ent, tets->s64.V,
                                                         prm->rho, s->mass);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(ctx, e, "lumped mass");
    s->rho = prm->rho;
  }
  BatchConst c;
  memset(&c, 0, sizeof c);
  c.nv = nv;
  c.dt = prm->dt;
  for (int k = 0; k < 3; ++k) c.g[k] = prm->gravity[k];
  c.rtol = prm->rtol;
  c.max_iters = prm->max_iters;
  const int nb = s->tb.nblocks;

  e = cudaMemsetAsync(s->sc, 0, (size_t)nmesh * sizeof(MeshCg), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->n_active, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "batched CG reset");
  // FP32 element operands are vertex-interleaved (see eidx).
  bool aos = false;
  if constexpr (sizeof(T) == 4) aos = mixed;
  if (aos)
    batch_prep_kernel<T, true><<<4 * 152, 256, 0, st>>>(nv, u, v, ue, pe, acc_f, acc_kv, acc_d, acc_kp, mixed);
  else
    batch_prep_kernel<T, false><<<4 * 152, 256, 0, st>>>(nv, u, v, ue, pe, acc_f, acc_kv, acc_d, acc_kp, mixed);
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
  if (aos)
    batch_init_kernel<T, true><<<nb, kBT, 0, st>>>(c, s->tb, pin, s->mass, acc_f, acc_kv, acc_d, s->r, s->p, s->y,
                                                   s->dinv, pe, s->part, s->sc, s->n_active);
  else
    batch_init_kernel<T, false><<<nb, kBT, 0, st>>>(c, s->tb, pin, s->mass, acc_f, acc_kv, acc_d, s->r, s->p, s->y,
                                                    s->dinv, mixed ? pe : nullptr, s->part, s->sc, s->n_active);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(ctx, e, "batched CG init");

  MapIO<T> kio;
  kio.u = io.u;
  kio.w = mixed ? pe : (const T*)s->p;
  kio.Kw = acc_kp;
  kio.aos = aos;
  // Capture kChunk iterations once; re-capture when anything baked in changes.
  std::vector<unsigned char> key(sizeof(BatchConst) + 5 * sizeof(double) + 3 * sizeof(void*));
  {
    unsigned char* k = key.data();
    memcpy(k, &c, sizeof c);
    k += sizeof c;
    const double kd[5] = {(double)sizeof(T), (double)prm->model, (double)prm->reduce, prm->mu + 1e-300 * prm->lambda,
                          (double)tets->layout_gen};
    memcpy(k, kd, sizeof kd);
    k += sizeof kd;
    const void* kp[3] = {pin, kio.u, kio.w};
    memcpy(k, kp, sizeof kp);
  }
  if (!s->chunk || s->key != key) {
    if (s->chunk) cudaGraphExecDestroy(s->chunk);
    s->chunk = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_check(ctx, e, "batched chunk capture");
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < kChunk && le == cudaSuccess; ++k) {
      const int par = k & 1;
      le = launch_tet_map<T>(tets, prm->model, OP_KV, prm->reduce, mu0, lam0, kio, s->n_active, st);
      if (aos)
        batch_pq_kernel<T, true><<<nb, kBT, 0, st>>>(c, s->tb, par, pin, s->mass, s->p, acc_kp, s->qz, s->part, s->sc,
                                                     s->n_active);
      else
        batch_pq_kernel<T, false><<<nb, kBT, 0, st>>>(c, s->tb, par, pin, s->mass, s->p, acc_kp, s->qz, s->part,
                                                      s->sc, s->n_active);
      batch_update_kernel<T><<<nb, kBT, 0, st>>>(c, s->tb, par, pin, s->p, s->dinv, s->r, s->y, s->qz, s->part,
                                                 s->sc, s->n_active);
      if (aos)
        batch_pupdate_kernel<T, true><<<nb, kBT, 0, st>>>(c, s->tb, par, pin, s->qz, s->p, pe, acc_kp, s->sc);
      else
        batch_pupdate_kernel<T, false><<<nb, kBT, 0, st>>>(c, s->tb, par, pin, s->qz, s->p, mixed ? pe : nullptr,
                                                           acc_kp, s->sc);
      if (le == cudaSuccess) le = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(st, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_check(ctx, le != cudaSuccess ? le : e, "batched chunk capture");
    }
    e = cudaGraphInstantiate(&s->chunk, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      s->chunk = nullptr;
      return cuda_check(ctx, e, "batched chunk instantiate");
    }
    s->key = key;
  }
  int launched = 0;
  while (true) {
    int h_active = 0;
    e = cudaGraphLaunch(s->chunk, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_active, s->n_active, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "batched CG chunk");
    launched += kChunk;
    if (h_active <= 0) break;
    if (launched > prm->max_iters + 2 * kChunk) break;  // defensive bound
  }
  batch_finish_kernel<<<4 * 152, 256, 0, st>>>(n, prm->dt, s->y, u, v);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->h_sc.data(), s->sc, (size_t)nmesh * sizeof(MeshCg), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_err, ctx->d_err, ERRW_WORDS * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "batched step finish");
  ebb_status_t status = EBB_OK;
  for (int m = 0; m < nmesh; ++m) {
    const MeshCg& h = s->h_sc[m];
    const double rel = h.bb > 0.0 ? std::sqrt(h.rr / h.bb) : 0.0;
    ebb_status_t ms = h.status;
    if (ms == EBB_OK && prm->fail_on_max_iters && h.iter >= prm->max_iters && rel > prm->rtol)
      ms = EBB_ERR_NOT_CONVERGED;
    if (reps) {
      reps[m].iters = h.iter;
      reps[m].rel_residual = rel;
      reps[m].status = ms;
    }
    if (ms != EBB_OK && status == EBB_OK) {
      status = ms;
      char buf[128];
      snprintf(buf, sizeof buf, "batch %d: %s", m,
               ms == EBB_ERR_CG_BREAKDOWN ? "PCG breakdown" : "PCG not converged");
      set_error(ctx, ms, buf);
    }
  }
  if (ctx->h_err[ERRW_CODE] != 0) {
    const int code = ctx->h_err[ERRW_CODE], idx = ctx->h_err[ERRW_INDEX];
    cudaMemsetAsync(ctx->d_err, 0, ERRW_WORDS * sizeof(int), st);
    cudaStreamSynchronize(st);
    char buf[128];
    snprintf(buf, sizeof buf, "device error %d at tet row %d", code, idx);
    status = set_error(ctx, code, buf);
  }
  return status;
}

}  // namespace

ebb_status_t run_batched_step(ebb_ctx_s* ctx, ebb_rel_s* tets, double* u, double* v, const void* pinned,
                              const int* batch, int nmesh, const ebb_step_params_t* p, ebb_cg_report_t* reps) {
  if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, EBB_ERR_CUDA, "cudaSetDevice failed");
  if (tets->vindex.off == nullptr) return set_error(ctx, EBB_ERR_STATE, "relation has no vertex index");
  ebb_status_t s = prepare_batch(ctx, tets, batch, nmesh);
  if (s) return s;
  return p->precision == EBB_PREC_F64
             ? batch_impl<double>(ctx, tets, u, v, (const unsigned char*)pinned, p, nmesh, reps)
             : batch_impl<float>(ctx, tets, u, v, (const unsigned char*)pinned, p, nmesh, reps);
}

}  // namespace ebb
