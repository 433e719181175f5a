// Assembled stiffness on the edge relation (block CSR) and its product with
// a vertex field.
//
// Section 5.2's tetmesh domain carries an edge relation with self-loops and
// a per-tet key-field tets.e[4][4] into it, and the Vega port of Section 7.2
// keeps the stiffness matrix on those edges, one 3x3 block per edge.  This
// file builds that structure over the internal vertex order: row r's blocks
// are (r, col[k]) for k in [row_off[r], row_off[r+1]), columns increasing,
// the diagonal block included; tet_blk[16 t + 4 a + b] (the tets.e[a][b]
// key) is the block of corners (a, b) of internal tet t.  The blocks are
// stored as 9 planes (entry (c, d) of block k at [(3 c + d) nnzb + k]), so
// that consecutive lanes reading consecutive blocks of a row read
// consecutive words.  K(x) is assembled from closed-form element blocks with
// atomic adds; K w is a block-sparse product with 8 lanes per row, each
// taking every 8th block of the row, and a fixed-order shuffle tree, so the
// product is bitwise reproducible for given blocks.
//
// Element block of corners a, b (b_a = row a-1 of Dm^-1, b_0 = minus their
// sum): the matrix-free K w map's dP applied to the probe dF = e_d b_b^T and
// contracted with b_a,
//   StVK: K_ab[c][d] = V (delta_cd b_b.S b_a + mu (F F^T)_cd b_a.b_b
//                         + mu r_b,c r_a,d + lam r_b,d r_a,c),     r_a = F b_a
//   NH:   K_ab[c][d] = V (mu delta_cd b_a.b_b + (mu - lam ln J) h_b,c h_a,d
//                         + lam h_b,d h_a,c),                      h_a = F^-T b_a.
#include <algorithm>
#include <vector>

#include "ebb_internal.h"
#include "tet_io.cuh"
#include "tet_math.cuh"

namespace ebb {

namespace {

constexpr int kAsmThreads = 128;
constexpr int kSpmvThreads = 256;

template <typename T, int MODEL, bool AOS>
__global__ void __launch_bounds__(kAsmThreads)
assemble_kernel(int nt, int nv, const int4* __restrict__ keys, const int* __restrict__ perm, TetStreams<T> s, T mu0,
                T lam0, MapIO<T> io, const int* __restrict__ tet_blk, int nnzb, T* blocks, int* err) {
  const int t = blockIdx.x * kAsmThreads + threadIdx.x;
  if (t >= nt) return;
  const int4 k4 = keys[t];
  const int kk[4] = {k4.x, k4.y, k4.z, k4.w};
  T B[9], V, mu, lam;
  load_tet(s, nt, t, mu0, lam0, B, V, mu, lam);
  T Du[9], Dw[9];
  load_edges<T, OP_FORCE, AOS>(io, nv, kk, Du, Dw);
  T G[9];
  mm(Du, B, G);
  T b[4][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    b[1][j] = B[j];
    b[2][j] = B[3 + j];
    b[3][j] = B[6 + j];
    b[0][j] = -(B[j] + B[3 + j] + B[6 + j]);
  }
  // Per corner: v_a (r_a for StVK, h_a for NH) and, for StVK, S b_a.
  T vec[4][3], Sb[4][3], FFt[9];
  T c1 = T(0);
  if (MODEL == EBB_STVK) {
    StvkState<T> sv;
    stvk_state(G, mu, lam, sv);
    T F[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) F[i] = G[i] + ((i % 4 == 0) ? T(1) : T(0));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        FFt[i * 3 + j] = F[i * 3 + 0] * F[j * 3 + 0] + F[i * 3 + 1] * F[j * 3 + 1] + F[i * 3 + 2] * F[j * 3 + 2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        vec[a][i] = F[i * 3 + 0] * b[a][0] + F[i * 3 + 1] * b[a][1] + F[i * 3 + 2] * b[a][2];
        Sb[a][i] = sv.S[i * 3 + 0] * b[a][0] + sv.S[i * 3 + 1] * b[a][1] + sv.S[i * 3 + 2] * b[a][2];
      }
  } else {
    NhState<T> sn;
    if (!nh_state(G, sn)) {
      raise_error(err, EBB_ERR_INVERTED, perm[t]);
      return;
    }
    c1 = mu - lam * sn.lnJ;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        vec[a][i] = sn.FiT[i * 3 + 0] * b[a][0] + sn.FiT[i * 3 + 1] * b[a][1] + sn.FiT[i * 3 + 2] * b[a][2];
  }
  const int* tb = tet_blk + (size_t)16 * t;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int bb = 0; bb < 4; ++bb) {
      const T bab = b[a][0] * b[bb][0] + b[a][1] * b[bb][1] + b[a][2] * b[bb][2];
      T* blk = blocks + tb[4 * a + bb];
      if (MODEL == EBB_STVK) {
        const T bSb = b[bb][0] * Sb[a][0] + b[bb][1] * Sb[a][1] + b[bb][2] * Sb[a][2];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const T k = (c == d ? bSb : T(0)) + mu * FFt[c * 3 + d] * bab + mu * vec[bb][c] * vec[a][d] +
                        lam * vec[bb][d] * vec[a][c];
            atomicAdd(blk + (size_t)(c * 3 + d) * nnzb, V * k);
          }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const T k = (c == d ? mu * bab : T(0)) + c1 * vec[bb][c] * vec[a][d] + lam * vec[bb][d] * vec[a][c];
            atomicAdd(blk + (size_t)(c * 3 + d) * nnzb, V * k);
          }
      }
    }
  }
}

// y[r] += sum_k blocks[k] w[col[k]] over row r's blocks; kRowLanes lanes per
// row, each taking every kRowLanes-th block of the row (8 measured faster
// than 4 and 16 on the 64^3 mesh's rows of about 15 blocks).
constexpr int kRowLanes = 8;

template <typename T, bool AOS>
__global__ void __launch_bounds__(kSpmvThreads)
bsr_spmv_kernel(int nv, int nnzb, const int* __restrict__ row_off, const int* __restrict__ col,
                const T* __restrict__ blocks, const T* __restrict__ w, T* y, const int* active) {
  if (active != nullptr && *active == 0) return;
  const int r = (int)((blockIdx.x * (unsigned)kSpmvThreads + threadIdx.x) / kRowLanes);
  const int l = threadIdx.x % kRowLanes;
  T acc[3] = {T(0), T(0), T(0)};
  if (r < nv) {
    const int k1 = row_off[r + 1];
#pragma unroll 2
    for (int k = row_off[r] + l; k < k1; k += kRowLanes) {
      const int j = col[k];
      T x[3];
      if constexpr (AOS) {
        const float4 q = reinterpret_cast<const float4*>(w)[j];
        x[0] = q.x;
        x[1] = q.y;
        x[2] = q.z;
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) x[c] = w[(size_t)c * nv + j];
      }
      const T* blk = blocks + k;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        acc[c] += blk[(size_t)(3 * c) * nnzb] * x[0] + blk[(size_t)(3 * c + 1) * nnzb] * x[1] +
                  blk[(size_t)(3 * c + 2) * nnzb] * x[2];
    }
  }
#pragma unroll
  for (int o = kRowLanes / 2; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, kRowLanes);
  if (r < nv && l == 0) {
    if constexpr (AOS) {
      float4* o = reinterpret_cast<float4*>(y) + r;
      float4 q = *o;
      q.x += (float)acc[0];
      q.y += (float)acc[1];
      q.z += (float)acc[2];
      *o = q;
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) y[(size_t)c * nv + r] += acc[c];
    }
  }
}

template <typename T>
const TetStreams<T>& tet_streams(const ebb_rel_s* rel);
template <>
const TetStreams<float>& tet_streams<float>(const ebb_rel_s* rel) { return rel->s32; }
template <>
const TetStreams<double>& tet_streams<double>(const ebb_rel_s* rel) { return rel->s64; }

cudaError_t upload_vec(int** dst, const std::vector<int>& v, cudaStream_t st) {
  cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(int));
  if (e == cudaSuccess && !v.empty()) e = cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(int),
                                                          cudaMemcpyHostToDevice, st);
  return e;
}

template <typename T, int MODEL>
cudaError_t launch_assemble_model(ebb_rel_s* rel, T mu0, T lam0, const MapIO<T>& io, T* blocks, cudaStream_t st) {
  const int nt = (int)rel->size, nv = (int)rel->verts->size;
  const TetStreams<T>& s = tet_streams<T>(rel);
  const int grid = (nt + kAsmThreads - 1) / kAsmThreads;
  if (io.aos) {
    if constexpr (sizeof(T) == 4)
      assemble_kernel<T, MODEL, true><<<grid, kAsmThreads, 0, st>>>(nt, nv, rel->keys, rel->tet_perm, s, mu0, lam0,
                                                                    io, rel->edges.tet_blk, rel->edges.nnzb, blocks,
                                                                    rel->ctx->d_err);
    else
      return cudaErrorInvalidValue;
  } else {
    assemble_kernel<T, MODEL, false><<<grid, kAsmThreads, 0, st>>>(nt, nv, rel->keys, rel->tet_perm, s, mu0, lam0,
                                                                   io, rel->edges.tet_blk, rel->edges.nnzb, blocks,
                                                                   rel->ctx->d_err);
  }
  return cudaGetLastError();
}

}  // namespace

ebb_status_t build_edges(ebb_ctx_s* ctx, ebb_rel_s* tets, const std::vector<int4>& keys) {
  const int nt = (int)keys.size();
  const int nv = (int)tets->verts->size;
  // vertex -> incident internal tets
  std::vector<int> voff((size_t)nv + 1, 0), vt((size_t)4 * nt);
  for (const int4& k : keys) {
    ++voff[(size_t)k.x + 1];
    ++voff[(size_t)k.y + 1];
    ++voff[(size_t)k.z + 1];
    ++voff[(size_t)k.w + 1];
  }
  for (int v = 0; v < nv; ++v) voff[v + 1] += voff[v];
  {
    std::vector<int> fill(voff.begin(), voff.end() - 1);
    for (int t = 0; t < nt; ++t) {
      const int k[4] = {keys[t].x, keys[t].y, keys[t].z, keys[t].w};
      for (int a = 0; a < 4; ++a) vt[fill[k[a]]++] = t;
    }
  }
  // rows: the distinct vertices of the tets around each vertex (itself included)
  std::vector<int> row_off((size_t)nv + 1, 0), col;
  col.reserve((size_t)nv * 16);
  std::vector<int> buf;
  for (int v = 0; v < nv; ++v) {
    buf.clear();
    buf.push_back(v);
    for (int i = voff[v]; i < voff[v + 1]; ++i) {
      const int4 k = keys[vt[i]];
      buf.push_back(k.x);
      buf.push_back(k.y);
      buf.push_back(k.z);
      buf.push_back(k.w);
    }
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    col.insert(col.end(), buf.begin(), buf.end());
    if (col.size() > (size_t)0x7fffffff / 9) return set_error(ctx, EBB_ERR_ARG, "edge relation too large");
    row_off[v + 1] = (int)col.size();
  }
  // tets.e[a][b]: the block of corners (a, b)
  std::vector<int> tb((size_t)16 * nt);
  for (int t = 0; t < nt; ++t) {
    const int k[4] = {keys[t].x, keys[t].y, keys[t].z, keys[t].w};
    for (int a = 0; a < 4; ++a) {
      const int* r0 = col.data() + row_off[k[a]];
      const int* r1 = col.data() + row_off[k[a] + 1];
      for (int b = 0; b < 4; ++b) tb[(size_t)16 * t + 4 * a + b] = (int)(std::lower_bound(r0, r1, k[b]) - col.data());
    }
  }
  EdgeIndex& E = tets->edges;
  E.nnzb = (int)col.size();
  cudaError_t e = upload_vec(&E.row_off, row_off, ctx->stream);
  if (e == cudaSuccess) e = upload_vec(&E.col, col, ctx->stream);
  if (e == cudaSuccess) e = upload_vec(&E.tet_blk, tb, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    free_edges(tets);
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, "device allocation for the edge relation failed");
  }
  return EBB_OK;
}

void free_edges(ebb_rel_s* tets) {
  EdgeIndex& E = tets->edges;
  cudaFree(E.row_off);
  cudaFree(E.col);
  cudaFree(E.tet_blk);
  cudaFree(E.blocks[0]);
  cudaFree(E.blocks[1]);
  for (int p = 0; p < 2; ++p) {
    cudaFree(E.rest[p]);
    cudaFree(E.qbuf[p]);
  }
  cudaFree(E.epart);
  E = EdgeIndex();
}

template <typename T>
cudaError_t launch_assemble(ebb_rel_s* rel, int model, T mu0, T lam0, const MapIO<T>& io, cudaStream_t st) {
  EdgeIndex& E = rel->edges;
  const int p = sizeof(T) == 4 ? 0 : 1;
  if (E.row_off == nullptr) return cudaErrorInvalidValue;
  if (E.blocks[p] == nullptr) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
    e = cudaMalloc(&E.blocks[p], std::max<size_t>(1, (size_t)E.nnzb) * 9 * sizeof(T));
    if (e != cudaSuccess) {
      E.blocks[p] = nullptr;
      return e;
    }
  }
  T* blocks = static_cast<T*>(E.blocks[p]);
  cudaError_t e = cudaMemsetAsync(blocks, 0, (size_t)E.nnzb * 9 * sizeof(T), st);
  if (e != cudaSuccess || rel->size == 0) {
    E.assembled[p] = e == cudaSuccess;
    return e;
  }
  e = model == EBB_STVK ? launch_assemble_model<T, EBB_STVK>(rel, mu0, lam0, io, blocks, st)
                        : launch_assemble_model<T, EBB_NEOHOOKEAN>(rel, mu0, lam0, io, blocks, st);
  E.assembled[p] = e == cudaSuccess;
  return e;
}

template <typename T>
cudaError_t launch_spmv(ebb_rel_s* rel, const T* w, T* y, bool aos, const int* active, cudaStream_t st) {
  const EdgeIndex& E = rel->edges;
  const int p = sizeof(T) == 4 ? 0 : 1;
  const int nv = (int)rel->verts->size;
  if (E.row_off == nullptr || !E.assembled[p]) return cudaErrorInvalidValue;
  if (nv == 0) return cudaSuccess;
  const int grid = (int)(((size_t)nv * kRowLanes + kSpmvThreads - 1) / kSpmvThreads);
  const T* blocks = static_cast<const T*>(E.blocks[p]);
  if (aos) {
    if constexpr (sizeof(T) == 4)
      bsr_spmv_kernel<T, true><<<grid, kSpmvThreads, 0, st>>>(nv, E.nnzb, E.row_off, E.col, blocks, w, y, active);
    else
      return cudaErrorInvalidValue;
  } else {
    bsr_spmv_kernel<T, false><<<grid, kSpmvThreads, 0, st>>>(nv, E.nnzb, E.row_off, E.col, blocks, w, y, active);
  }
  return cudaGetLastError();
}

template cudaError_t launch_assemble<float>(ebb_rel_s*, int, float, float, const MapIO<float>&, cudaStream_t);
template cudaError_t launch_assemble<double>(ebb_rel_s*, int, double, double, const MapIO<double>&, cudaStream_t);
template cudaError_t launch_spmv<float>(ebb_rel_s*, const float*, float*, bool, const int*, cudaStream_t);
template cudaError_t launch_spmv<double>(ebb_rel_s*, const double*, double*, bool, const int*, cudaStream_t);

}  // namespace ebb
