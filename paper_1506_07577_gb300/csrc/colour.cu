// Vertex-conflict colouring of the tets relation for the atomic-free
// reduction variant.
//
// Tets of one colour share no vertex, so a map restricted to one colour can
// reduce into vertex fields with plain read-modify-write; colours run one
// after another on the stream, which makes the result independent of thread
// scheduling (bitwise reproducible).  This is the colouring approach to
// reductions that Section 7.4 attributes to Liszt, kept beside the atomic
// variant of Section 6.2.  Colouring is greedy (first-fit in tet order) on the
// host; tets are then stored colour by colour (stable within a colour).
#include <cstdint>
#include <cstdio>
#include <vector>

#include "ebb_internal.h"

namespace ebb {

namespace {

constexpr int kMaxColourWords = 4;  // up to 256 colours

template <typename T>
__global__ void gather_planes_kernel(int n, int planes, const int* __restrict__ perm, const T* __restrict__ src,
                                     T* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int o = perm[i];
  for (int p = 0; p < planes; ++p) dst[(size_t)p * n + i] = src[(size_t)p * n + o];
}

__global__ void gather_keys_kernel(int n, const int* __restrict__ perm, const int4* __restrict__ src, int4* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[perm[i]];
}

template <typename T>
cudaError_t gather_copy(int n, int planes, const int* perm, const T* src, T** dst, cudaStream_t st) {
  if (!src) return cudaSuccess;
  cudaError_t e = cudaMalloc(dst, sizeof(T) * (size_t)planes * n);
  if (e != cudaSuccess) return e;
  gather_planes_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(n, planes, perm, src, *dst);
  return cudaGetLastError();
}

}  // namespace

void free_colouring(ebb_rel_s* tets) {
  Colouring& c = tets->colour;
  cudaFree(c.keys);
  cudaFree(c.perm);
  cudaFree(c.s64.B);
  cudaFree(c.s64.V);
  cudaFree(c.s64.mu);
  cudaFree(c.s64.lam);
  cudaFree(c.s32.B);
  cudaFree(c.s32.V);
  cudaFree(c.s32.mu);
  cudaFree(c.s32.lam);
  tets->colour = Colouring();
  tets->has_colour = false;
}

ebb_status_t build_colouring(ebb_ctx_s* ctx, ebb_rel_s* tets) {
  free_colouring(tets);
  const int nt = (int)tets->size;
  const int nv = (int)tets->verts->size;
  cudaStream_t st = ctx->stream;
  std::vector<int4> hk(nt);
  cudaError_t e = cudaMemcpyAsync(hk.data(), tets->keys, sizeof(int4) * nt, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "colouring: reading keys");

  std::vector<uint64_t> used((size_t)nv * kMaxColourWords, 0);
  std::vector<int> colour(nt);
  int ncol = 0;
  for (int t = 0; t < nt; ++t) {
    const int k[4] = {hk[t].x, hk[t].y, hk[t].z, hk[t].w};
    int c = -1;
    for (int w = 0; w < kMaxColourWords && c < 0; ++w) {
      uint64_t m = 0;
      for (int a = 0; a < 4; ++a) m |= used[(size_t)k[a] * kMaxColourWords + w];
      if (~m) c = w * 64 + __builtin_ctzll(~m);
    }
    if (c < 0) return set_error(ctx, EBB_ERR_ARG, "colouring needs more than 256 colours");
    colour[t] = c;
    for (int a = 0; a < 4; ++a) used[(size_t)k[a] * kMaxColourWords + c / 64] |= 1ull << (c % 64);
    if (c + 1 > ncol) ncol = c + 1;
  }
  std::vector<int> offsets(ncol + 1, 0);
  for (int t = 0; t < nt; ++t) offsets[colour[t] + 1]++;
  for (int c = 0; c < ncol; ++c) offsets[c + 1] += offsets[c];
  std::vector<int> perm(nt), fill(offsets.begin(), offsets.end() - 1);
  for (int t = 0; t < nt; ++t) perm[fill[colour[t]]++] = t;

  int* dperm = nullptr;
  Colouring& col = tets->colour;
  e = cudaMalloc(&dperm, sizeof(int) * nt);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMalloc(&col.keys, sizeof(int4) * nt);
  if (e == cudaSuccess) {
    gather_keys_kernel<<<(nt + 255) / 256, 256, 0, st>>>(nt, dperm, tets->keys, col.keys);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = gather_copy(nt, 1, dperm, tets->tet_perm, &col.perm, st);
  if (e == cudaSuccess) e = gather_copy(nt, 9, dperm, tets->s64.B, &col.s64.B, st);
  if (e == cudaSuccess) e = gather_copy(nt, 1, dperm, tets->s64.V, &col.s64.V, st);
  if (e == cudaSuccess) e = gather_copy(nt, 1, dperm, tets->s64.mu, &col.s64.mu, st);
  if (e == cudaSuccess) e = gather_copy(nt, 1, dperm, tets->s64.lam, &col.s64.lam, st);
  if (e == cudaSuccess) e = gather_copy(nt, 9, dperm, tets->s32.B, &col.s32.B, st);
  if (e == cudaSuccess) e = gather_copy(nt, 1, dperm, tets->s32.V, &col.s32.V, st);
  if (e == cudaSuccess) e = gather_copy(nt, 1, dperm, tets->s32.mu, &col.s32.mu, st);
  if (e == cudaSuccess) e = gather_copy(nt, 1, dperm, tets->s32.lam, &col.s32.lam, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dperm);
  if (e != cudaSuccess) {
    free_colouring(tets);
    return cuda_check(ctx, e, "colouring: building coloured copies");
  }
  col.ncolours = ncol;
  col.offsets = offsets;
  tets->has_colour = true;
  return EBB_OK;
}

}  // namespace ebb
