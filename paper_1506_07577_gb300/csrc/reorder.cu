// Vertex renumbering (EBB_FINALIZE_REORDER_VERTS) and staging of map
// operands in the vertex-interleaved layout.
//
// Keys are opaque (Section 5.1 and its footnote), so the library may number
// vertices its own way: Morton order of the rest positions, which puts the
// vertices of neighbouring tets next to each other in memory.  Caller-owned
// vertex fields keep the caller's order; these kernels move values between
// the two orders (the permutation is a bijection, so scatters never
// collide).
#include <algorithm>
#include <cstdint>
#include <tuple>
#include <vector>

#include "ebb_internal.h"

namespace ebb {
namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void gather_kernel(int nv, const int* __restrict__ vperm, const T* __restrict__ src, T* dst) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= nv) return;
  const int o = vperm[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) dst[(size_t)c * nv + i] = src[(size_t)c * nv + o];
}

template <typename T>
__global__ void scatter_add_kernel(int nv, const int* __restrict__ vperm, const T* __restrict__ src, T* dst) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= nv) return;
  const int o = vperm[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) dst[(size_t)c * nv + o] += src[(size_t)c * nv + i];
}

__global__ void scatter_kernel(int nv, const int* __restrict__ vperm, const double* __restrict__ src, double* dst) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= nv) return;
  const int o = vperm[i];
#pragma unroll
  for (int c = 0; c < 3; ++c) dst[(size_t)c * nv + o] = src[(size_t)c * nv + i];
}

template <typename PT>
__global__ void gather_pin_kernel(int nv, const int* __restrict__ vperm, const PT* __restrict__ src,
                                  unsigned char* dst) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= nv) return;
  dst[i] = src == nullptr ? 0 : (src[vperm[i]] != 0 ? 1 : 0);
}

// dst_k[4 i + c] = src_k[c][o(i)] (padding 0), o = vperm or identity, for
// one or two fields.
__global__ void interleave_kernel(int nv, const int* __restrict__ vperm, const float* __restrict__ a,
                                  const float* __restrict__ b, float4* __restrict__ da, float4* __restrict__ db) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= nv) return;
  const int o = vperm ? vperm[i] : i;
  da[i] = make_float4(a[o], a[(size_t)nv + o], a[2 * (size_t)nv + o], 0.f);
  if (b) db[i] = make_float4(b[o], b[(size_t)nv + o], b[2 * (size_t)nv + o], 0.f);
}

// dst_k[c][o(i)] += src_k[4 i + c] for up to three fields.
__global__ void deinterleave_add_kernel(int nv, const int* __restrict__ vperm, const float4* __restrict__ s0,
                                        float* d0, const float4* __restrict__ s1, float* d1,
                                        const float4* __restrict__ s2, float* d2) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= nv) return;
  const size_t o = vperm ? vperm[i] : i;
  const float4* src[3] = {s0, s1, s2};
  float* dst[3] = {d0, d1, d2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (!src[k]) continue;
    const float4 x = src[k][i];
    dst[k][o] += x.x;
    dst[k][(size_t)nv + o] += x.y;
    dst[k][2 * (size_t)nv + o] += x.z;
  }
}

__global__ void permute_vec4_kernel(int nv, const int* __restrict__ vperm, const float4* __restrict__ src,
                                    float4* __restrict__ dst) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i < nv) dst[i] = src[vperm[i]];
}

__global__ void permute_add_vec4_kernel(int nv, const int* __restrict__ vperm, const float4* __restrict__ src,
                                        float4* dst) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= nv) return;
  const float4 s = src[i];
  float4 d = dst[vperm[i]];
  d.x += s.x;
  d.y += s.y;
  d.z += s.z;
  dst[vperm[i]] = d;
}

uint64_t spread3(uint64_t x) {
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

// Rows [r0, r1) of packed (x, y, z) triples to 4-float elements (x, y, z, 0)
// and back, for one field or two: the host-buffer map's transfers in 12-byte
// rows (blocks striding over the rows).
constexpr int kXyzThreads = 256;
constexpr int kXyzMaxBlocks = 4 * 152;

__global__ void xyz_to_x4_kernel(int r0, int r1, const float* __restrict__ sa, const float* __restrict__ sb,
                                 float4* __restrict__ da, float4* __restrict__ db) {
  for (int r = r0 + blockIdx.x * kXyzThreads + threadIdx.x; r < r1; r += gridDim.x * kXyzThreads) {
    const float* p = sa + 3 * (size_t)r;
    da[r] = make_float4(p[0], p[1], p[2], 0.f);
    if (sb) {
      const float* q = sb + 3 * (size_t)r;
      db[r] = make_float4(q[0], q[1], q[2], 0.f);
    }
  }
}

__global__ void x4_to_xyz_kernel(int r0, int r1, const float4* __restrict__ sa, const float4* __restrict__ sb,
                                 float* __restrict__ da, float* __restrict__ db) {
  for (int r = r0 + blockIdx.x * kXyzThreads + threadIdx.x; r < r1; r += gridDim.x * kXyzThreads) {
    const float4 a = sa[r];
    float* p = da + 3 * (size_t)r;
    p[0] = a.x;
    p[1] = a.y;
    p[2] = a.z;
    if (sb) {
      const float4 b = sb[r];
      float* q = db + 3 * (size_t)r;
      q[0] = b.x;
      q[1] = b.y;
      q[2] = b.z;
    }
  }
}

int xyz_blocks(int rows) { return std::max(1, std::min((rows + kXyzThreads - 1) / kXyzThreads, kXyzMaxBlocks)); }

}  // namespace

cudaError_t xyz_to_x4(const float* sa, const float* sb, float* da, float* db, int r0, int r1, cudaStream_t st) {
  if (r1 <= r0) return cudaSuccess;
  xyz_to_x4_kernel<<<xyz_blocks(r1 - r0), kXyzThreads, 0, st>>>(r0, r1, sa, sb, (float4*)da, (float4*)db);
  return cudaGetLastError();
}

cudaError_t x4_to_xyz(const float* sa, const float* sb, float* da, float* db, int r0, int r1, cudaStream_t st) {
  if (r1 <= r0) return cudaSuccess;
  x4_to_xyz_kernel<<<xyz_blocks(r1 - r0), kXyzThreads, 0, st>>>(r0, r1, (const float4*)sa, (const float4*)sb, da,
                                                                  db);
  return cudaGetLastError();
}

template <typename T>
cudaError_t gather_vertex_field(int nv, const int* vperm, const T* src, T* dst, cudaStream_t st) {
  if (nv == 0) return cudaSuccess;
  gather_kernel<T><<<(nv + kThreads - 1) / kThreads, kThreads, 0, st>>>(nv, vperm, src, dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t scatter_add_vertex_field(int nv, const int* vperm, const T* src, T* dst, cudaStream_t st) {
  if (nv == 0) return cudaSuccess;
  scatter_add_kernel<T><<<(nv + kThreads - 1) / kThreads, kThreads, 0, st>>>(nv, vperm, src, dst);
  return cudaGetLastError();
}

cudaError_t scatter_vertex_field(int nv, const int* vperm, const double* src, double* dst, cudaStream_t st) {
  if (nv == 0) return cudaSuccess;
  scatter_kernel<<<(nv + kThreads - 1) / kThreads, kThreads, 0, st>>>(nv, vperm, src, dst);
  return cudaGetLastError();
}

template <typename PT>
cudaError_t gather_pinned(int nv, const int* vperm, const PT* src, unsigned char* dst, cudaStream_t st) {
  if (nv == 0) return cudaSuccess;
  gather_pin_kernel<PT><<<(nv + kThreads - 1) / kThreads, kThreads, 0, st>>>(nv, vperm, src, dst);
  return cudaGetLastError();
}

cudaError_t permute_vec4(int nv, const int* vperm, const float* src, float* dst, cudaStream_t st) {
  if (nv == 0) return cudaSuccess;
  permute_vec4_kernel<<<(nv + kThreads - 1) / kThreads, kThreads, 0, st>>>(nv, vperm, (const float4*)src,
                                                                          (float4*)dst);
  return cudaGetLastError();
}

cudaError_t permute_add_vec4(int nv, const int* vperm, const float* src, float* dst, cudaStream_t st) {
  if (nv == 0) return cudaSuccess;
  permute_add_vec4_kernel<<<(nv + kThreads - 1) / kThreads, kThreads, 0, st>>>(nv, vperm, (const float4*)src,
                                                                              (float4*)dst);
  return cudaGetLastError();
}

cudaError_t interleave_fields(int nv, const int* vperm, const float* a, const float* b, float* da, float* db,
                              cudaStream_t st) {
  if (nv == 0) return cudaSuccess;
  interleave_kernel<<<(nv + kThreads - 1) / kThreads, kThreads, 0, st>>>(nv, vperm, a, b, (float4*)da, (float4*)db);
  return cudaGetLastError();
}

cudaError_t deinterleave_add_fields(int nv, const int* vperm, const float* const* src, float* const* dst, int n,
                                    cudaStream_t st) {
  if (nv == 0 || n == 0) return cudaSuccess;
  const float4* s[3] = {nullptr, nullptr, nullptr};
  float* d[3] = {nullptr, nullptr, nullptr};
  for (int k = 0; k < n && k < 3; ++k) {
    s[k] = (const float4*)src[k];
    d[k] = dst[k];
  }
  deinterleave_add_kernel<<<(nv + kThreads - 1) / kThreads, kThreads, 0, st>>>(nv, vperm, s[0], d[0], s[1], d[1],
                                                                             s[2], d[2]);
  return cudaGetLastError();
}

template cudaError_t gather_vertex_field<float>(int, const int*, const float*, float*, cudaStream_t);
template cudaError_t gather_vertex_field<double>(int, const int*, const double*, double*, cudaStream_t);
template cudaError_t scatter_add_vertex_field<float>(int, const int*, const float*, float*, cudaStream_t);
template cudaError_t scatter_add_vertex_field<double>(int, const int*, const double*, double*, cudaStream_t);
template cudaError_t gather_pinned<unsigned char>(int, const int*, const unsigned char*, unsigned char*,
                                                  cudaStream_t);
template cudaError_t gather_pinned<int>(int, const int*, const int*, unsigned char*, cudaStream_t);

void vertex_morton_order(const std::vector<double>& X, std::vector<int>& perm) {
  const int nv = (int)(X.size() / 3);
  double lo[3], hi[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = nv ? *std::min_element(X.begin() + (size_t)c * nv, X.begin() + (size_t)(c + 1) * nv) : 0.0;
    hi[c] = nv ? *std::max_element(X.begin() + (size_t)c * nv, X.begin() + (size_t)(c + 1) * nv) : 1.0;
    if (!(hi[c] > lo[c])) hi[c] = lo[c] + 1.0;
  }
  const double q = (double)((1u << 21) - 1);
  std::vector<uint64_t> code(nv);
  for (int v = 0; v < nv; ++v) {
    uint64_t m = 0;
    for (int c = 0; c < 3; ++c) {
      double r = (X[(size_t)c * nv + v] - lo[c]) / (hi[c] - lo[c]);
      r = r < 0 ? 0 : (r > 1 ? 1 : r);
      m |= spread3((uint64_t)(r * q)) << c;
    }
    code[v] = m;
  }
  perm.clear();
  radix_order(code, 63, perm);  // by code, ties by vertex number
}

}  // namespace ebb
