// C ABI entry points: contexts, relations, fields, finalize and map calls.
//
// The runtime side of Ebb's relational model (Section 6.1): relations are
// row counts with column-store fields bound to them; a key-field links tets
// to vertices (Section 5.1); finalize validates keys (accesses cannot go out
// of bounds, Section 5.1) and precomputes the per-tet rest-shape data the
// maps read.  The phase rule of Section 4.1 is enforced per map call: a
// field that a map reduces into may not also be read by it.
#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ebb_internal.h"

using namespace ebb;

namespace ebb {

ebb_status_t set_error(ebb_ctx_s* ctx, ebb_status_t code, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

ebb_status_t cuda_check(ebb_ctx_s* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return EBB_OK;
  return set_error(ctx, EBB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace ebb

namespace {

size_t dtype_size(ebb_dtype_t d) {
  switch (d) {
    case EBB_F32: return 4;
    case EBB_F64: return 8;
    case EBB_I32: return 4;
    case EBB_U8: return 1;
    case EBB_F32X4: return 4;
  }
  return 0;
}

// Rest-shape precomputation: B = Dm^-1 and V = det(Dm)/6 in FP64, plus FP32
// copies.  Dm = [X1-X0, X2-X0, X3-X0] with X read through the keys.
__global__ void rest_shape_kernel(int nt, int nv, const int4* __restrict__ keys, const int* __restrict__ perm,
                                  const double* __restrict__ X, double* B64, double* V64, float* B32, float* V32,
                                  int* err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int4 k = keys[t];
  const int kk[4] = {k.x, k.y, k.z, k.w};
  double D[9];
  for (int c = 0; c < 3; ++c) {
    const double x0 = X[(size_t)c * nv + kk[0]];
    for (int j = 0; j < 3; ++j) D[c * 3 + j] = X[(size_t)c * nv + kk[j + 1]] - x0;
  }
  const double c00 = D[4] * D[8] - D[5] * D[7];
  const double c01 = D[5] * D[6] - D[3] * D[8];
  const double c02 = D[3] * D[7] - D[4] * D[6];
  const double det = D[0] * c00 + D[1] * c01 + D[2] * c02;
  if (!(det > 0.0)) {
    if (atomicCAS(err + ERRW_CODE, 0, EBB_ERR_INVERTED) == 0) err[ERRW_INDEX] = perm[t];
  }
  const double id = 1.0 / det;
  // inverse = adj / det, adj = cof^T
  double Bm[9];
  Bm[0] = c00 * id;
  Bm[3] = c01 * id;
  Bm[6] = c02 * id;
  Bm[1] = (D[2] * D[7] - D[1] * D[8]) * id;
  Bm[4] = (D[0] * D[8] - D[2] * D[6]) * id;
  Bm[7] = (D[1] * D[6] - D[0] * D[7]) * id;
  Bm[2] = (D[1] * D[5] - D[2] * D[4]) * id;
  Bm[5] = (D[2] * D[3] - D[0] * D[5]) * id;
  Bm[8] = (D[0] * D[4] - D[1] * D[3]) * id;
  for (int i = 0; i < 9; ++i) {
    B64[(size_t)i * nt + t] = Bm[i];
    B32[(size_t)i * nt + t] = (float)Bm[i];
  }
  V64[t] = det / 6.0;
  V32[t] = (float)(det / 6.0);
}

// Per-tet Lame parameters gathered into the internal tet order.
__global__ void copy_material_kernel(int nt, const int* __restrict__ perm, const double* __restrict__ mu,
                                     const double* __restrict__ lam, double* mu64, double* lam64, float* mu32,
                                     float* lam32) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int o = perm[t];
  const double m = mu[o], l = lam[o];
  mu64[t] = m;
  lam64[t] = l;
  mu32[t] = (float)m;
  lam32[t] = (float)l;
}

void free_host_plan(ebb_rel_s* r) {
  HostPlan* p = r->hplan;
  if (!p) return;
  for (int c = 0; c < HostPlan::kChunks; ++c) {
    if (p->ev_in[c]) cudaEventDestroy(p->ev_in[c]);
    if (p->ev_map[c]) cudaEventDestroy(p->ev_map[c]);
  }
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->ev_end) cudaEventDestroy(p->ev_end);
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_out) cudaStreamDestroy(p->s_out);
  delete p;
  r->hplan = nullptr;
}

void free_tet_data(ebb_rel_s* r) {
  free_host_plan(r);
  cudaFree(r->xyz_stage);
  r->xyz_stage = nullptr;
  cudaFree(r->keys);
  r->keys = nullptr;
  cudaFree(r->vperm);
  r->vperm = nullptr;
  r->vorder.clear();
  r->vown = -1;
  for (void*& p : r->vscratch) {
    cudaFree(p);
    p = nullptr;
  }
  for (void*& p : r->gather_corner) {
    cudaFree(p);
    p = nullptr;
  }
  cudaFree(r->s64.B);
  cudaFree(r->s64.V);
  cudaFree(r->s64.mu);
  cudaFree(r->s64.lam);
  cudaFree(r->s32.B);
  cudaFree(r->s32.V);
  cudaFree(r->s32.mu);
  cudaFree(r->s32.lam);
  r->s64 = TetStreams<double>();
  r->s32 = TetStreams<float>();
  free_colouring(r);
  free_edges(r);
  free_layout(r);
  free_step_scratch(r);
  free_batch_scratch(r);
  r->finalized = false;
}

const Field* find_field(const ebb_rel_s* r, const char* name) {
  if (!r || !name) return nullptr;
  auto it = r->fields.find(name);
  return it == r->fields.end() ? nullptr : &it->second;
}

ebb_status_t read_device_error(ebb_ctx_s* ctx) {
  cudaError_t e = cudaMemcpyAsync(ctx->h_err, ctx->d_err, ERRW_WORDS * sizeof(int), cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "reading device status");
  const int code = ctx->h_err[ERRW_CODE];
  if (code == 0) return EBB_OK;
  const int idx = ctx->h_err[ERRW_INDEX];
  cudaMemsetAsync(ctx->d_err, 0, ERRW_WORDS * sizeof(int), ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  char buf[160];
  if (code == EBB_ERR_INVERTED)
    snprintf(buf, sizeof buf, "inverted element (det <= 0) at tet row %d", idx);
  else if (code == EBB_ERR_KEY)
    snprintf(buf, sizeof buf, "key out of range at row %d", idx);
  else if (code == EBB_ERR_TIMEOUT)
    snprintf(buf, sizeof buf, "bounded device wait timed out (site %d)", idx);
  else
    snprintf(buf, sizeof buf, "device error %d at index %d", code, idx);
  return set_error(ctx, code, buf);
}

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

// A concrete reduction variant (AUTO resolved).
bool valid_reduce(int r) {
  return r == EBB_REDUCE_ATOMIC || r == EBB_REDUCE_COLOR || r == EBB_REDUCE_TILED || r == EBB_REDUCE_GATHER ||
         r == EBB_REDUCE_TILED_ORDERED || r == EBB_REDUCE_COOP;
}

// EBB_REDUCE_AUTO: the autotuned variant for this model and precision, else
// the tiled one.
ebb_reduce_t resolve_reduce(const ebb_rel_s* tets, ebb_reduce_t r, int model, int precision) {
  if (r != EBB_REDUCE_AUTO) return r;
  if ((model == EBB_STVK || model == EBB_NEOHOOKEAN) && (precision == EBB_PREC_F64 || precision == EBB_PREC_F32)) {
    const int t = tets->tuned[model][precision];
    if (t >= 0) return (ebb_reduce_t)t;
  }
  return EBB_REDUCE_TILED;
}

// Resolve a vertex field used by a map or step; checks dtype and width.
ebb_status_t vertex_field(ebb_ctx_s* ctx, ebb_rel_s* tets, const char* name, ebb_dtype_t want, int ncomp,
                          void** out) {
  if (!name) return set_error(ctx, EBB_ERR_ARG, "null field name");
  const Field* f = find_field(tets->verts, name);
  if (!f) return set_error(ctx, EBB_ERR_ARG, std::string("no vertex field named '") + name + "'");
  if (f->dtype != want || f->ncomp != ncomp)
    return set_error(ctx, EBB_ERR_ARG, std::string("vertex field '") + name + "' has the wrong dtype or width");
  *out = f->ptr;
  return EBB_OK;
}

struct MapCall {
  const char* in[2] = {nullptr, nullptr};
  const char* out[3] = {nullptr, nullptr, nullptr};
  int nin = 0, nout = 0;
};

// One entry point for the four map calls.
// Resolve the vertex fields of one map call: F64 planes, or F32 as all
// planes or all EBB_F32X4 elements (*x4 reports which).
ebb_status_t map_fields(ebb_ctx_s* ctx, ebb_rel_s* tets, const char* const* names, int n, bool f64, void** out,
                        bool* x4) {
  *x4 = false;
  for (int i = 0; i < n; ++i) {
    if (!names[i]) return set_error(ctx, EBB_ERR_ARG, "null field name");
    const Field* f = find_field(tets->verts, names[i]);
    if (!f) return set_error(ctx, EBB_ERR_ARG, std::string("no vertex field named '") + names[i] + "'");
    const bool ok = f->ncomp == 3 && (f64 ? f->dtype == EBB_F64 : (f->dtype == EBB_F32 || f->dtype == EBB_F32X4));
    if (!ok)
      return set_error(ctx, EBB_ERR_ARG, std::string("vertex field '") + names[i] + "' has the wrong dtype or width");
    const bool fx4 = f->dtype == EBB_F32X4;
    if (i == 0) *x4 = fx4;
    if (fx4 != *x4) return set_error(ctx, EBB_ERR_ARG, "a map's F32 fields must all be planes or all EBB_F32X4");
    out[i] = f->ptr;
  }
  return EBB_OK;
}

// Launch a map on caller-layout (3-plane) device fields: FP32 tiled maps on
// a relation the autotuner set to stage, or with reordered vertices, move
// their operands into library-owned vertex-interleaved buffers and add the
// results back; relations with reordered vertices stage in the internal order;
// otherwise the map runs on the caller's fields directly.  Outputs are `+=`
// targets in every case.
ebb_status_t launch_map_staged(ebb_ctx_s* ctx, ebb_rel_s* tets, int ops, int model, double mu, double lambda,
                               ebb_reduce_t reduce, bool f64, bool x4, void* const* in_user, int nin,
                               void* const* out_user, int nout, bool drop) {
  const int nv = (int)tets->verts->size;
  const size_t bytes = (size_t)nv * (x4 ? 16 : 3 * (f64 ? 8 : 4));
  // Reordered vertices are staged anyway, so their FP32 tiled maps always
  // stage interleaved.  EBB_F32X4 fields are interleaved already.
  const bool stage = !x4 && !f64 && (reduce == EBB_REDUCE_TILED || reduce == EBB_REDUCE_TILED_ORDERED) &&
                     (tets->stage_interleaved || tets->vperm != nullptr);
  void* in[2] = {in_user[0], nin > 1 ? in_user[1] : nullptr};
  void* out[3] = {nullptr, nullptr, nullptr};
  for (int i = 0; i < nout; ++i) out[i] = out_user[i];
  if (stage || tets->vperm) {   // (EBB_F32X4 fields with reordered vertices are permuted as whole elements)
    for (int i = 0; i < 5; ++i)   // 3 nv doubles: holds either precision and the interleaved FP32 layout
      if (!tets->vscratch[i] && cudaMalloc(&tets->vscratch[i], (size_t)nv * 3 * 8 + 16) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, EBB_ERR_NOMEM, "device allocation for staged map operands failed");
      }
    cudaError_t ge = cudaSuccess;
    if (x4) {
      for (int i = 0; i < nin && ge == cudaSuccess; ++i) {
        ge = permute_vec4(nv, tets->vperm, (const float*)in[i], (float*)tets->vscratch[i], ctx->stream);
        in[i] = tets->vscratch[i];
      }
    } else if (stage) {
      ge = interleave_fields(nv, tets->vperm, (const float*)in[0], (const float*)in[1], (float*)tets->vscratch[0],
                             (float*)tets->vscratch[1], ctx->stream);
      in[0] = tets->vscratch[0];
      if (nin > 1) in[1] = tets->vscratch[1];
    } else {
      for (int i = 0; i < nin && ge == cudaSuccess; ++i) {
        ge = f64 ? gather_vertex_field<double>(nv, tets->vperm, (const double*)in[i], (double*)tets->vscratch[i],
                                               ctx->stream)
                 : gather_vertex_field<float>(nv, tets->vperm, (const float*)in[i], (float*)tets->vscratch[i],
                                              ctx->stream);
        in[i] = tets->vscratch[i];
      }
    }
    for (int i = 0; i < nout && ge == cudaSuccess; ++i) {
      out[i] = tets->vscratch[2 + i];
      ge = cudaMemsetAsync(out[i], 0, (stage || x4) ? (size_t)nv * 16 : bytes, ctx->stream);
    }
    if (ge != cudaSuccess) return cuda_check(ctx, ge, "staging map operands");
  }
  cudaError_t e;
  int oi = 0;
  if (f64) {
    MapIO<double> io;
    io.u = (const double*)in[0];
    io.w = (const double*)in[1];
    if (ops & OP_FORCE) io.f = (double*)out[oi++];
    if (ops & (OP_KV | OP_SPMV)) io.Kw = (double*)out[oi++];
    if (ops & OP_DIAG) io.d = (double*)out[oi++];
    tets->test_drop_tile = drop ? 0 : -1;
    e = launch_tet_map<double>(tets, model, ops, reduce, mu, lambda, io, nullptr, ctx->stream);
    tets->test_drop_tile = -1;
  } else {
    MapIO<float> io;
    io.u = (const float*)in[0];
    io.w = (const float*)in[1];
    if (ops & OP_FORCE) io.f = (float*)out[oi++];
    if (ops & (OP_KV | OP_SPMV)) io.Kw = (float*)out[oi++];
    if (ops & OP_DIAG) io.d = (float*)out[oi++];
    io.aos = stage || x4;
    tets->test_drop_tile = drop ? 0 : -1;
    e = launch_tet_map<float>(tets, model, ops, reduce, (float)mu, (float)lambda, io, nullptr, ctx->stream);
    tets->test_drop_tile = -1;
  }
  if (e == cudaSuccess && x4 && tets->vperm) {
    for (int i = 0; i < nout && e == cudaSuccess; ++i)
      e = permute_add_vec4(nv, tets->vperm, (const float*)out[i], (float*)out_user[i], ctx->stream);
  } else if (e == cudaSuccess && stage) {
    e = deinterleave_add_fields(nv, tets->vperm, (const float* const*)out, (float* const*)out_user, nout,
                                ctx->stream);
  } else if (e == cudaSuccess && tets->vperm) {
    for (int i = 0; i < nout && e == cudaSuccess; ++i)
      e = f64 ? scatter_add_vertex_field<double>(nv, tets->vperm, (const double*)out[i], (double*)out_user[i],
                                                 ctx->stream)
              : scatter_add_vertex_field<float>(nv, tets->vperm, (const float*)out[i], (float*)out_user[i],
                                                ctx->stream);
  }
  return cuda_check(ctx, e, "launching tet map");
}

ebb_status_t run_map(ebb_ctx_t ctx, ebb_rel_t tets, const MapCall& mc, int ops, const ebb_map_opts_t* opts) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (!tets || !opts) return set_error(ctx, EBB_ERR_ARG, "null relation or options");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  if (opts->model != EBB_STVK && opts->model != EBB_NEOHOOKEAN)
    return set_error(ctx, EBB_ERR_ARG, "unknown material model");
  if (opts->precision != EBB_PREC_F64 && opts->precision != EBB_PREC_F32)
    return set_error(ctx, EBB_ERR_ARG, "unknown precision");
  const ebb_reduce_t reduce = resolve_reduce(tets, opts->reduce, opts->model, opts->precision);
  if (!valid_reduce(reduce))
    return set_error(ctx, EBB_ERR_ARG, "unknown reduction variant");
  if (reduce == EBB_REDUCE_COLOR && !tets->has_colour)
    return set_error(ctx, EBB_ERR_STATE, "colour reduction requested but relation finalized without EBB_FINALIZE_COLOR");
  const bool f64 = opts->precision == EBB_PREC_F64;
  void* in[2] = {nullptr, nullptr};
  void* out[3] = {nullptr, nullptr, nullptr};
  const char* names[5];
  void* ptrs[5];
  for (int i = 0; i < mc.nin; ++i) names[i] = mc.in[i];
  for (int i = 0; i < mc.nout; ++i) names[mc.nin + i] = mc.out[i];
  bool x4 = false;
  {
    ebb_status_t s = map_fields(ctx, tets, names, mc.nin + mc.nout, f64, ptrs, &x4);
    if (s) return s;
  }
  for (int i = 0; i < mc.nin; ++i) in[i] = ptrs[i];
  for (int i = 0; i < mc.nout; ++i) out[i] = ptrs[mc.nin + i];
  const size_t bytes = (size_t)tets->verts->size * (x4 ? 16 : 3 * (f64 ? 8 : 4));
  // Phase rule: a reduce target may not be read by the same map, nor be
  // reduced into twice.
  for (int i = 0; i < mc.nout; ++i) {
    for (int j = 0; j < mc.nin; ++j)
      if (ranges_overlap(out[i], bytes, in[j], bytes))
        return set_error(ctx, EBB_ERR_PHASE, std::string("field '") + mc.out[i] +
                                                 "' is both reduced into and read by one map");
    for (int j = i + 1; j < mc.nout; ++j)
      if (ranges_overlap(out[i], bytes, out[j], bytes))
        return set_error(ctx, EBB_ERR_PHASE, "two reduce targets of one map overlap");
  }
  const bool drop = (opts->flags & EBB_MAP_TEST_DROP_TILE) != 0;
  if (drop && reduce != EBB_REDUCE_TILED)
    return set_error(ctx, EBB_ERR_ARG, "EBB_MAP_TEST_DROP_TILE needs the tiled reduction");
  if (opts->flags & EBB_MAP_ZERO_OUT) {
    for (int i = 0; i < mc.nout; ++i) {
      ebb_status_t s = cuda_check(ctx, cudaMemsetAsync(out[i], 0, bytes, ctx->stream), "zeroing output");
      if (s) return s;
    }
  }
  return launch_map_staged(ctx, tets, ops, opts->model, opts->mu, opts->lambda, reduce, f64, x4, in, mc.nin, out,
                           mc.nout, drop);
}

}  // namespace

extern "C" {

ebb_status_t ebb_ctx_create(ebb_ctx_t* out, int device, void* cuda_stream) {
  if (!out) return EBB_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return EBB_ERR_ARG;
  ebb_ctx_s* ctx = new (std::nothrow) ebb_ctx_s();
  if (!ctx) return EBB_ERR_NOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&ctx->d_err, ERRW_WORDS * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_err, ERRW_WORDS * sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_err, 0, ERRW_WORDS * sizeof(int)) != cudaSuccess) {
    cudaFree(ctx->d_err);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    delete ctx;
    return EBB_ERR_CUDA;
  }
  *out = ctx;
  return EBB_OK;
}

ebb_status_t ebb_ctx_set_stream(ebb_ctx_t ctx, void* cuda_stream) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->stream = (cudaStream_t)cuda_stream;
  return EBB_OK;
}

ebb_status_t ebb_ctx_destroy(ebb_ctx_t ctx) {
  if (!ctx) return EBB_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (ebb_rel_s* r : ctx->rels) {
    free_tet_data(r);
    delete r;
  }
  cudaFree(ctx->d_err);
  cudaFreeHost(ctx->h_err);
  delete ctx;
  return EBB_OK;
}

ebb_status_t ebb_ctx_sync(ebb_ctx_t ctx) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  return read_device_error(ctx);
}

const char* ebb_last_error(ebb_ctx_t ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

ebb_status_t ebb_relation_create(ebb_ctx_t ctx, const char* name, int64_t size, ebb_rel_t* out) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (!out || !name) return set_error(ctx, EBB_ERR_ARG, "null name or output");
  if (size < 0 || size > (int64_t)0x7fffffff / 9)
    return set_error(ctx, EBB_ERR_ARG, "relation size out of range [0, 2^31/9)");
  ebb_rel_s* r = new (std::nothrow) ebb_rel_s();
  if (!r) return set_error(ctx, EBB_ERR_NOMEM, "out of host memory");
  r->ctx = ctx;
  r->name = name;
  r->size = size;
  ctx->rels.push_back(r);
  *out = r;
  return EBB_OK;
}

ebb_status_t ebb_field_bind(ebb_rel_t rel, const char* name, ebb_dtype_t dtype, int32_t ncomp, void* device_ptr,
                            ebb_rel_t key_target) {
  if (!rel) return EBB_ERR_ARG;
  ebb_ctx_s* ctx = rel->ctx;
  ctx->last_error.clear();
  if (!name || !*name) return set_error(ctx, EBB_ERR_ARG, "empty field name");
  if (dtype_size(dtype) == 0) return set_error(ctx, EBB_ERR_ARG, "unknown dtype");
  if (ncomp < 1 || ncomp > 16) return set_error(ctx, EBB_ERR_ARG, "ncomp out of range [1,16]");
  if (!device_ptr && rel->size > 0) return set_error(ctx, EBB_ERR_ARG, "null device pointer");
  if (key_target && dtype != EBB_I32) return set_error(ctx, EBB_ERR_ARG, "key-fields must be I32");
  if (dtype == EBB_F32X4 && (ncomp != 3 || ((uintptr_t)device_ptr & 15u) != 0))
    return set_error(ctx, EBB_ERR_ARG, "EBB_F32X4 fields need ncomp 3 and a 16-byte aligned pointer");
  if (key_target && key_target->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "key target in another context");
  Field f;
  f.name = name;
  f.dtype = dtype;
  f.ncomp = ncomp;
  f.ptr = device_ptr;
  f.key_target = key_target;
  rel->fields[name] = f;
  return EBB_OK;
}

static ebb_status_t relation_finalize(ebb_rel_t tets, uint32_t flags) {
  ebb_ctx_s* ctx = tets->ctx;
  ctx->last_error.clear();
  const Field* kv = find_field(tets, "v");
  if (!kv || kv->dtype != EBB_I32 || kv->ncomp != 4 || !kv->key_target)
    return set_error(ctx, EBB_ERR_ARG, "tets needs key-field 'v' (I32, 4 components, key target = verts)");
  ebb_rel_s* verts = kv->key_target;
  const Field* X = find_field(verts, "X");
  if (!X || X->dtype != EBB_F64 || X->ncomp != 3)
    return set_error(ctx, EBB_ERR_ARG, "verts needs field 'X' (F64, 3 components): rest positions");
  const Field* fmu = find_field(tets, "mu");
  const Field* flam = find_field(tets, "lambda");
  if ((fmu != nullptr) != (flam != nullptr))
    return set_error(ctx, EBB_ERR_ARG, "bind both 'mu' and 'lambda' per tet, or neither");
  if (fmu && (fmu->dtype != EBB_F64 || fmu->ncomp != 1 || flam->dtype != EBB_F64 || flam->ncomp != 1))
    return set_error(ctx, EBB_ERR_ARG, "per-tet 'mu'/'lambda' must be F64 with 1 component");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, EBB_ERR_CUDA, "cudaSetDevice failed");

  free_tet_data(tets);
  if (cudaError_t pe = prepare_map_kernels()) return cuda_check(ctx, pe, "configuring map kernels");
  tets->verts = verts;
  const int nt = (int)tets->size;
  const int nv = (int)verts->size;
  if (nt == 0) {
    // Still build the (empty) vertex index: the lumped mass reads it.
    std::vector<int4> none, sorted;
    std::vector<int> perm;
    std::vector<unsigned char> prefix;
    ebb_status_t ls =
        build_layout(ctx, tets, none, std::vector<double>((size_t)3 * nv, 0.0), nullptr, perm, sorted, prefix);
    if (!ls && (flags & EBB_FINALIZE_EDGES)) ls = build_edges(ctx, tets, none);
    if (ls) return ls;
    tets->finalized = true;
    return EBB_OK;
  }

  // Keys: validate on the host (accesses through keys can then never leave
  // the target relation) and repack as one int4 per tet.
  std::vector<int> hk((size_t)nt * 4);
  ebb_status_t s = cuda_check(ctx, cudaMemcpyAsync(hk.data(), kv->ptr, hk.size() * sizeof(int),
                                                   cudaMemcpyDeviceToHost, ctx->stream),
                              "copying keys");
  if (s) return s;
  s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "copying keys");
  if (s) return s;
  std::vector<int4> packed(nt);
  for (int t = 0; t < nt; ++t) {
    int k[4];
    for (int a = 0; a < 4; ++a) {
      k[a] = hk[(size_t)a * nt + t];
      if (k[a] < 0 || k[a] >= nv) {
        char buf[128];
        snprintf(buf, sizeof buf, "key out of range at tet row %d corner %d (value %d, %d vertices)", t, a, k[a], nv);
        return set_error(ctx, EBB_ERR_KEY, buf);
      }
    }
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (k[a] == k[b]) {
          char buf[128];
          snprintf(buf, sizeof buf, "tet row %d repeats vertex %d", t, k[a]);
          return set_error(ctx, EBB_ERR_KEY, buf);
        }
    packed[t] = make_int4(k[0], k[1], k[2], k[3]);
  }
  // Rest positions on the host for the Morton order of the tets.
  std::vector<double> hX((size_t)3 * nv);
  s = cuda_check(ctx, cudaMemcpyAsync(hX.data(), X->ptr, hX.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                      ctx->stream),
                 "copying rest positions");
  if (s) return s;
  s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "copying rest positions");
  if (s) return s;
  // Optional per-vertex group ids ("batch", I32): tets are then ordered by
  // group first, and a tet may not join vertices of two groups.
  std::vector<int> hbatch;
  if (const Field* fb = find_field(verts, "batch")) {
    if (fb->dtype != EBB_I32 || fb->ncomp != 1)
      return set_error(ctx, EBB_ERR_ARG, "verts.batch must be I32 with 1 component");
    hbatch.resize(nv);
    s = cuda_check(ctx, cudaMemcpyAsync(hbatch.data(), fb->ptr, (size_t)nv * sizeof(int), cudaMemcpyDeviceToHost,
                                        ctx->stream),
                   "copying batch ids");
    if (s) return s;
    s = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "copying batch ids");
    if (s) return s;
    for (int t = 0; t < nt; ++t) {
      const int b = hbatch[packed[t].x];
      if (b < 0 || hbatch[packed[t].y] != b || hbatch[packed[t].z] != b || hbatch[packed[t].w] != b) {
        char buf[128];
        snprintf(buf, sizeof buf, "tet row %d joins vertices of different batches (or a negative batch id)", t);
        return set_error(ctx, EBB_ERR_KEY, buf);
      }
    }
  }
  // Optional vertex renumbering: keys, rest positions and everything built
  // from them switch to the internal (Morton) vertex order.  REORDER keeps
  // the vertex fields in the caller's order (maps and steps stage them);
  // RENUMBER makes the new order the relation's own, for every vertex field
  // bound or read from now on.
  double* X_int = nullptr;
  std::vector<int> tperm;
  const bool renumber = (flags & EBB_FINALIZE_RENUMBER_VERTS) != 0;
  if ((flags & EBB_FINALIZE_REORDER_VERTS) && renumber)
    return set_error(ctx, EBB_ERR_ARG, "EBB_FINALIZE_REORDER_VERTS and EBB_FINALIZE_RENUMBER_VERTS exclude each other");
  if ((flags & EBB_FINALIZE_REORDER_VERTS) || renumber) {
    if (!hbatch.empty())
      return set_error(ctx, EBB_ERR_ARG, "renumbering vertices cannot be combined with verts.batch");
    std::vector<int> vp, vinv(nv);
    if (renumber) {
      // The Morton order of the tets depends on their centroids only, which
      // renumbering the vertices leaves as they are: build_layout reuses it.
      // rows grouped by the chunks of the host-buffer map (Morton-ordered
      // tets cut into tiles), so that its copies of one chunk's rows
      // overlap the map of another
      int own = nv;
      chunked_vertex_order(packed, hX, tets->tile_cap, HostPlan::kChunks, vp, &own, &tperm);
      tets->vown = own;
    } else {
      vertex_morton_order(hX, vp);
    }
    for (int i = 0; i < nv; ++i) vinv[vp[i]] = i;
    for (int t = 0; t < nt; ++t)
      packed[t] = make_int4(vinv[packed[t].x], vinv[packed[t].y], vinv[packed[t].z], vinv[packed[t].w]);
    std::vector<double> hXi(hX.size());
    for (int c = 0; c < 3; ++c)
      for (int i = 0; i < nv; ++i) hXi[(size_t)c * nv + i] = hX[(size_t)c * nv + vp[i]];
    hX.swap(hXi);
    cudaError_t ve = cudaSuccess;
    if (renumber) {
      tets->vorder = vp;
    } else {
      ve = cudaMalloc(&tets->vperm, sizeof(int) * nv);
      if (ve == cudaSuccess) ve = cudaMemcpy(tets->vperm, vp.data(), sizeof(int) * nv, cudaMemcpyHostToDevice);
    }
    if (ve == cudaSuccess) ve = cudaMalloc(&X_int, sizeof(double) * hX.size());
    if (ve == cudaSuccess) ve = cudaMemcpy(X_int, hX.data(), sizeof(double) * hX.size(), cudaMemcpyHostToDevice);
    if (ve != cudaSuccess) {
      cudaFree(X_int);
      free_tet_data(tets);
      cudaGetLastError();
      return set_error(ctx, EBB_ERR_NOMEM, "device allocation for the vertex order failed");
    }
  }
  std::vector<int> perm;
  std::vector<int4> sorted;
  std::vector<unsigned char> prefix;
  s = build_layout(ctx, tets, packed, hX, hbatch.empty() ? nullptr : &hbatch, perm, sorted, prefix,
                   tperm.empty() ? nullptr : &tperm);
  if (s) {
    cudaFree(X_int);
    return s;
  }
  packed.swap(sorted);

  cudaError_t e = cudaMalloc(&tets->keys, sizeof(int4) * nt);
  if (e == cudaSuccess) e = cudaMalloc(&tets->s64.B, sizeof(double) * 9 * nt);
  if (e == cudaSuccess) e = cudaMalloc(&tets->s64.V, sizeof(double) * nt);
  if (e == cudaSuccess) e = cudaMalloc(&tets->s32.B, sizeof(float) * 9 * nt);
  if (e == cudaSuccess) e = cudaMalloc(&tets->s32.V, sizeof(float) * nt);
  if (e == cudaSuccess && fmu) {
    e = cudaMalloc(&tets->s64.mu, sizeof(double) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&tets->s64.lam, sizeof(double) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&tets->s32.mu, sizeof(float) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&tets->s32.lam, sizeof(float) * nt);
  }
  if (e != cudaSuccess) {
    cudaFree(X_int);
    free_tet_data(tets);
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, "device allocation for tet data failed");
  }
  e = cudaMemcpyAsync(tets->keys, packed.data(), sizeof(int4) * nt, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    const int th = 256, gr = (nt + th - 1) / th;
    const double* Xk = X_int ? X_int : (const double*)X->ptr;
    rest_shape_kernel<<<gr, th, 0, ctx->stream>>>(nt, nv, tets->keys, tets->tet_perm, Xk, tets->s64.B,
                                                  tets->s64.V, tets->s32.B, tets->s32.V, ctx->d_err);
    if (fmu)
      copy_material_kernel<<<gr, th, 0, ctx->stream>>>(nt, tets->tet_perm, (const double*)fmu->ptr,
                                                       (const double*)flam->ptr, tets->s64.mu, tets->s64.lam,
                                                       tets->s32.mu, tets->s32.lam);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(X_int);
  if (e != cudaSuccess) {
    free_tet_data(tets);
    return cuda_check(ctx, e, "rest-shape precomputation");
  }
  s = read_device_error(ctx);
  if (s) {
    free_tet_data(tets);
    return s;
  }
  s = build_tile_blobs(ctx, tets, prefix);
  if (s) {
    free_tet_data(tets);
    return s;
  }
  if (flags & EBB_FINALIZE_COLOR) {
    s = build_colouring(ctx, tets);
    if (s) {
      free_tet_data(tets);
      return s;
    }
  }
  if (flags & EBB_FINALIZE_EDGES) {
    s = build_edges(ctx, tets, packed);
    if (s) {
      free_tet_data(tets);
      return s;
    }
  }
  tets->finalized = true;
  return EBB_OK;
}

// Re-tiling, with host memory that runs out (an exception of the set-up
// code) as a status; the tiles may then be gone, so the relation has to be
// finalized again.
static ebb_status_t retile(ebb_ctx_s* ctx, ebb_rel_s* tets, int cap) {
  try {
    return rebuild_tiles(ctx, tets, cap);
  } catch (const std::bad_alloc&) {
    free_tet_data(tets);
    tets->finalized = false;
    return set_error(ctx, EBB_ERR_NOMEM, "host memory for the tile tables ran out; finalize the relation again");
  }
}

// Host memory for the layout (keys, orders, tile tables) runs out as an
// exception of the set-up code; it becomes a status here.
ebb_status_t ebb_relation_finalize(ebb_rel_t tets, uint32_t flags) {
  if (!tets) return EBB_ERR_ARG;
  try {
    return relation_finalize(tets, flags);
  } catch (const std::bad_alloc&) {
    free_tet_data(tets);
    return set_error(tets->ctx, EBB_ERR_NOMEM, "host memory for the tet layout ran out");
  }
}

ebb_status_t ebb_map_tet_forces(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* f_out,
                                const ebb_map_opts_t* opts) {
  MapCall mc;
  mc.in[0] = u;
  mc.nin = 1;
  mc.out[0] = f_out;
  mc.nout = 1;
  return run_map(ctx, tets, mc, OP_FORCE, opts);
}

ebb_status_t ebb_map_tet_Kv(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* w, const char* Kw_out,
                            const ebb_map_opts_t* opts) {
  MapCall mc;
  mc.in[0] = u;
  mc.in[1] = w;
  mc.nin = 2;
  mc.out[0] = Kw_out;
  mc.nout = 1;
  return run_map(ctx, tets, mc, OP_KV, opts);
}

ebb_status_t ebb_map_tet_force_Kv(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* w, const char* f_out,
                                  const char* Kw_out, const ebb_map_opts_t* opts) {
  MapCall mc;
  mc.in[0] = u;
  mc.in[1] = w;
  mc.nin = 2;
  mc.out[0] = f_out;
  mc.out[1] = Kw_out;
  mc.nout = 2;
  return run_map(ctx, tets, mc, OP_FORCE | OP_KV, opts);
}

extern "C++" {
namespace {

// The chunk plan of `tets` for its current tiles (built on first use and
// after the tiles change).
ebb_status_t host_plan(ebb_ctx_s* ctx, ebb_rel_s* tets, HostPlan** out) {
  HostPlan* p = tets->hplan;
  if (p && p->gen == tets->layout_gen) {
    *out = p;
    return EBB_OK;
  }
  if (!p) {
    p = new HostPlan();
    tets->hplan = p;
    cudaError_t e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_end, cudaEventDisableTiming);
    for (int c = 0; c < HostPlan::kChunks && e == cudaSuccess; ++c) {
      e = cudaEventCreateWithFlags(&p->ev_in[c], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_map[c], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      free_host_plan(tets);
      return cuda_check(ctx, e, "host-map streams");
    }
  }
  const Tiles& tl = tets->tiles;
  const int nt = (int)tets->size, nv = (int)tets->verts->size, ntiles = tl.ntiles;
  std::vector<int4> hdr(ntiles), keys(nt);
  cudaError_t e = cudaMemcpy2DAsync(hdr.data(), sizeof(int4), tl.blob32, tl.L32.bytes, sizeof(int4), ntiles,
                                    cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(keys.data(), tets->keys, sizeof(int4) * nt, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "host-map plan");
  const int K = std::min(HostPlan::kChunks, ntiles);
  p->K = K;
  p->tile_off.assign(K + 1, 0);
  p->need_hi.assign(K, 0);
  p->done_lo.assign(K, nv);
  // per chunk: the lowest and one past the highest row below `own` it touches
  const int own0 = tets->vown >= 0 ? tets->vown : nv;
  std::vector<int> lo_own(K, own0), hi_own(K, 0);
  for (int c = 0; c < K; ++c) {
    p->tile_off[c + 1] = chunk_first_tile(c + 1, ntiles, K);
    const int r0 = hdr[p->tile_off[c]].z;
    const int r1 = hdr[p->tile_off[c + 1] - 1].z + hdr[p->tile_off[c + 1] - 1].x;
    for (int t = r0; t < r1; ++t) {
      const int k4[4] = {keys[t].x, keys[t].y, keys[t].z, keys[t].w};
      for (int a = 0; a < 4; ++a)
        if (k4[a] < own0) {
          lo_own[c] = std::min(lo_own[c], k4[a]);
          hi_own[c] = std::max(hi_own[c], k4[a] + 1);
        }
    }
  }
  // Rows from `own` on (the vertices several chunks share, on a relation
  // that renumbered its vertices by chunk) go in before the first chunk and
  // out after the last; the ranges below cover the rows before them.
  const int own = tets->vown >= 0 ? tets->vown : nv;
  p->own = own;
  for (int c = 0; c < K; ++c) {
    p->need_hi[c] = std::max(c > 0 ? p->need_hi[c - 1] : 0, std::min(hi_own[c], own));
    p->done_lo[c] = own;
  }
  for (int c = K - 2; c >= 0; --c) p->done_lo[c] = std::min(p->done_lo[c + 1], lo_own[c + 1]);
  p->gen = tets->layout_gen;
  *out = p;
  return EBB_OK;
}

// Rows [r0, r1) of one vertex field between host and device buffers, as one
// copy (EBB_F32X4) or one per plane.
cudaError_t copy_rows(void* dst, const void* src, int r0, int r1, int nv, bool x4, size_t elem, cudaMemcpyKind kind,
                      cudaStream_t st) {
  if (r1 <= r0) return cudaSuccess;
  if (x4) return cudaMemcpyAsync((char*)dst + 16 * (size_t)r0, (const char*)src + 16 * (size_t)r0,
                                 16 * (size_t)(r1 - r0), kind, st);
  for (int c = 0; c < 3; ++c) {
    const size_t off = ((size_t)c * nv + r0) * elem;
    cudaError_t e = cudaMemcpyAsync((char*)dst + off, (const char*)src + off, (size_t)(r1 - r0) * elem, kind, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Rows [r0, r1) of an input field from the host, and of an output field to
// the host: as copy_rows, or, with a staging buffer (EBB_MAP_HOST_XYZ), as
// packed (x, y, z) host rows that pass through `stage` on the device and are
// widened to (or narrowed from) the field's 4-float elements there.
cudaError_t rows_in(void* dev, const void* host, float* stage, int r0, int r1, int nv, bool x4, size_t elem,
                    cudaStream_t st) {
  if (!stage) return copy_rows(dev, host, r0, r1, nv, x4, elem, cudaMemcpyHostToDevice, st);
  if (r1 <= r0) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(stage + 3 * (size_t)r0, (const float*)host + 3 * (size_t)r0,
                                  12 * (size_t)(r1 - r0), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = xyz_to_x4(stage, nullptr, (float*)dev, nullptr, r0, r1, st);
  return e;
}
cudaError_t rows_out(void* host, const void* dev, float* stage, int r0, int r1, int nv, bool x4, size_t elem,
                     cudaStream_t st) {
  if (!stage) return copy_rows(host, dev, r0, r1, nv, x4, elem, cudaMemcpyDeviceToHost, st);
  if (r1 <= r0) return cudaSuccess;
  cudaError_t e = x4_to_xyz((const float*)dev, nullptr, stage, nullptr, r0, r1, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((float*)host + 3 * (size_t)r0, stage + 3 * (size_t)r0, 12 * (size_t)(r1 - r0),
                        cudaMemcpyDeviceToHost, st);
  return e;
}

// The host-buffer map in tile chunks: chunk c's input rows are copied in on
// one stream, its tiles mapped on the context's stream once they have
// landed, and the output rows it completes copied out on a third stream,
// so that the copies of one chunk overlap the map of another.
template <typename T>
ebb_status_t host_map_chunked(ebb_ctx_s* ctx, ebb_rel_s* tets, void* const* dev, bool x4, bool same_input,
                              const void* u_host, const void* w_host, void* f_host, void* Kw_host, float* stage,
                              const ebb_map_opts_t* opts, ebb_reduce_t reduce) {
  HostPlan* P = nullptr;
  ebb_status_t s = host_plan(ctx, tets, &P);
  if (s) return s;
  const int nv = (int)tets->verts->size;
  const size_t bytes = (size_t)nv * (x4 ? 16 : 3 * sizeof(T));
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaEventRecord(P->ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s_in, P->ev_start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s_out, P->ev_start, 0);
  if (e == cudaSuccess && (opts->flags & EBB_MAP_ZERO_OUT)) {
    e = cudaMemsetAsync(dev[2], 0, bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev[3], 0, bytes, st);
  }
  MapIO<T> io;
  io.u = (const T*)dev[0];
  io.w = (const T*)dev[1];
  io.f = (T*)dev[2];
  io.Kw = (T*)dev[3];
  io.aos = x4;
  // Packed host rows (EBB_MAP_HOST_XYZ) pass through the staging buffer:
  // the copy streams move 12-byte rows between the host and the staging,
  // and the rows a chunk reads are widened into the fields just before its
  // map, the rows it completes narrowed just after, on the map's stream
  // (kernels beside the map would find its SMs full).  Without staging the
  // copies move the fields' own rows.
  const size_t sn = 3 * (size_t)nv;
  float* const stg[4] = {stage, stage ? stage + sn : nullptr, stage ? stage + 2 * sn : nullptr,
                         stage ? stage + 3 * sn : nullptr};
  float* const w_dev = same_input ? nullptr : (float*)dev[1];
  float* const w_stg = same_input ? nullptr : stg[1];
  auto packed_copy = [&](void* dst, const void* src, int r0, int r1, cudaMemcpyKind kind, cudaStream_t cs) {
    if (r1 <= r0) return cudaSuccess;
    return cudaMemcpyAsync((float*)dst + 3 * (size_t)r0, (const float*)src + 3 * (size_t)r0, 12 * (size_t)(r1 - r0),
                           kind, cs);
  };
  auto copy_in = [&](int r0, int r1) {
    cudaError_t ce = stage ? packed_copy(stg[0], u_host, r0, r1, cudaMemcpyHostToDevice, P->s_in)
                           : copy_rows(dev[0], u_host, r0, r1, nv, x4, sizeof(T), cudaMemcpyHostToDevice, P->s_in);
    if (ce == cudaSuccess && !same_input)
      ce = stage ? packed_copy(stg[1], w_host, r0, r1, cudaMemcpyHostToDevice, P->s_in)
                 : copy_rows(dev[1], w_host, r0, r1, nv, x4, sizeof(T), cudaMemcpyHostToDevice, P->s_in);
    return ce;
  };
  auto copy_out = [&](int r0, int r1) {
    cudaError_t ce = stage ? packed_copy(f_host, stg[2], r0, r1, cudaMemcpyDeviceToHost, P->s_out)
                 : copy_rows(f_host, dev[2], r0, r1, nv, x4, sizeof(T), cudaMemcpyDeviceToHost, P->s_out);
    if (ce == cudaSuccess)
      ce = stage ? packed_copy(Kw_host, stg[3], r0, r1, cudaMemcpyDeviceToHost, P->s_out)
                 : copy_rows(Kw_host, dev[3], r0, r1, nv, x4, sizeof(T), cudaMemcpyDeviceToHost, P->s_out);
    return ce;
  };
  // the shared rows first
  if (e == cudaSuccess) e = copy_in(P->own, nv);
  int in_done = 0, out_done = 0;
  for (int c = 0; c < P->K && e == cudaSuccess; ++c) {
    e = copy_in(in_done, P->need_hi[c]);
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_in[c], P->s_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P->ev_in[c], 0);
    if (stage) {
      if (e == cudaSuccess && c == 0) e = xyz_to_x4(stg[0], w_stg, (float*)dev[0], w_dev, P->own, nv, st);
      if (e == cudaSuccess) e = xyz_to_x4(stg[0], w_stg, (float*)dev[0], w_dev, in_done, P->need_hi[c], st);
    }
    in_done = P->need_hi[c];
    io.tile_begin = P->tile_off[c];
    io.tile_end = P->tile_off[c + 1];
    if (e == cudaSuccess)
      e = launch_tet_map<T>(tets, opts->model, OP_FORCE | OP_KV, reduce, (T)opts->mu, (T)opts->lambda, io, nullptr, st);
    if (e == cudaSuccess && stage)
      e = x4_to_xyz((const float*)dev[2], (const float*)dev[3], stg[2], stg[3], out_done, P->done_lo[c], st);
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_map[c], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s_out, P->ev_map[c], 0);
    if (e == cudaSuccess) e = copy_out(out_done, P->done_lo[c]);
    out_done = P->done_lo[c];
  }
  // the rows before `own` that no chunk touched, and the shared rows, last
  // (narrowed after the last map; its event is recorded again)
  if (e == cudaSuccess && stage) {
    e = x4_to_xyz((const float*)dev[2], (const float*)dev[3], stg[2], stg[3], out_done, nv, st);
    if (e == cudaSuccess) e = cudaEventRecord(P->ev_map[P->K - 1], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->s_out, P->ev_map[P->K - 1], 0);
  }
  if (e == cudaSuccess) e = copy_out(out_done, nv);
  if (e == cudaSuccess) e = cudaEventRecord(P->ev_end, P->s_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, P->ev_end, 0);
  if (e != cudaSuccess) return cuda_check(ctx, e, "chunked host-buffer map");
  // Waits for the last copies and reports any device-detected error.
  return read_device_error(ctx);
}

}  // namespace
}  // extern "C++"

ebb_status_t ebb_map_tet_force_Kv_host(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* w,
                                       const char* f_out, const char* Kw_out, const void* u_host,
                                       const void* w_host, void* f_host, void* Kw_host,
                                       const ebb_map_opts_t* opts) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (!tets || !opts) return set_error(ctx, EBB_ERR_ARG, "null relation or options");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  if (opts->precision != EBB_PREC_F64 && opts->precision != EBB_PREC_F32)
    return set_error(ctx, EBB_ERR_ARG, "unknown precision");
  // Resolve the fields and apply the map's checks before copying anything.
  const bool f64 = opts->precision == EBB_PREC_F64;
  const char* names[4] = {u, w, f_out, Kw_out};
  void* dev[4];
  bool x4 = false;
  ebb_status_t s = map_fields(ctx, tets, names, 4, f64, dev, &x4);
  if (s) return s;
  const size_t bytes = (size_t)tets->verts->size * (x4 ? 16 : 3 * (f64 ? 8 : 4));
  for (int o = 2; o < 4; ++o) {
    if (ranges_overlap(dev[o], bytes, dev[0], bytes) || ranges_overlap(dev[o], bytes, dev[1], bytes))
      return set_error(ctx, EBB_ERR_PHASE, std::string("field '") + names[o] +
                                               "' is both reduced into and read by one map");
  }
  if (ranges_overlap(dev[2], bytes, dev[3], bytes))
    return set_error(ctx, EBB_ERR_PHASE, "two reduce targets of one map overlap");
  if (bytes > 0 && (!u_host || !w_host || !f_host || !Kw_host))
    return set_error(ctx, EBB_ERR_ARG, "null host buffer");
  // Both input copies land in the bound fields: if u and w overlap on the
  // device, the second copy would overwrite the first, unless they are one
  // field filled from one host buffer.
  const bool same_input = dev[0] == dev[1] && u_host == w_host;
  if (ranges_overlap(dev[0], bytes, dev[1], bytes) && !same_input)
    return set_error(ctx, EBB_ERR_PHASE, "fields u and w overlap on the device but come from different host buffers");
  if (opts->model != EBB_STVK && opts->model != EBB_NEOHOOKEAN)
    return set_error(ctx, EBB_ERR_ARG, "unknown material model");
  // Packed (x, y, z) host rows: staged on the device, widened into and
  // narrowed from the 4-float fields there.
  const bool xyz = (opts->flags & EBB_MAP_HOST_XYZ) != 0;
  if (xyz && (!x4 || f64))
    return set_error(ctx, EBB_ERR_ARG, "EBB_MAP_HOST_XYZ needs FP32 fields of EBB_F32X4 elements");
  float* stage = nullptr;
  if (xyz && bytes > 0) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, EBB_ERR_CUDA, "cudaSetDevice failed");
    if (!tets->xyz_stage && cudaMalloc(&tets->xyz_stage, sizeof(float) * 12 * (size_t)tets->verts->size) != cudaSuccess) {
      tets->xyz_stage = nullptr;
      cudaGetLastError();
      return set_error(ctx, EBB_ERR_NOMEM, "device allocation for the packed-row staging failed");
    }
    stage = tets->xyz_stage;
  }
  // The tiled map on fields it reads in place runs in chunks that overlap
  // the copies; every other form copies everything in, maps, copies out.
  const ebb_reduce_t reduce = resolve_reduce(tets, opts->reduce, opts->model, opts->precision);
  const bool staged = !x4 && !f64 && tets->stage_interleaved;
  if (bytes > 0 && reduce == EBB_REDUCE_TILED && !tets->vperm && !staged &&
      !(opts->flags & EBB_MAP_TEST_DROP_TILE) && tets->tiles.ntiles >= 2 * HostPlan::kChunks) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(ctx, EBB_ERR_CUDA, "cudaSetDevice failed");
    return f64 ? host_map_chunked<double>(ctx, tets, dev, x4, same_input, u_host, w_host, f_host, Kw_host, stage,
                                          opts, reduce)
               : host_map_chunked<float>(ctx, tets, dev, x4, same_input, u_host, w_host, f_host, Kw_host, stage,
                                         opts, reduce);
  }
  cudaError_t e = cudaSuccess;
  const int nv = (int)tets->verts->size;
  const size_t elem = f64 ? 8 : 4, sn = 3 * (size_t)nv;
  if (bytes > 0) {
    e = rows_in(dev[0], u_host, stage, 0, nv, nv, x4, elem, ctx->stream);
    if (e == cudaSuccess && !same_input)
      e = rows_in(dev[1], w_host, stage ? stage + sn : nullptr, 0, nv, nv, x4, elem, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "copying u, w to the device");
  }
  s = ebb_map_tet_force_Kv(ctx, tets, u, w, f_out, Kw_out, opts);
  if (s) return s;
  if (bytes > 0) {
    e = rows_out(f_host, dev[2], stage ? stage + 2 * sn : nullptr, 0, nv, nv, x4, elem, ctx->stream);
    if (e == cudaSuccess)
      e = rows_out(Kw_host, dev[3], stage ? stage + 3 * sn : nullptr, 0, nv, nv, x4, elem, ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "copying f, Kw to the host");
  }
  // Waits for the copies and reports any device-detected error of the map.
  return read_device_error(ctx);
}

ebb_status_t ebb_map_tet_diagK(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* d_out,
                               const ebb_map_opts_t* opts) {
  MapCall mc;
  mc.in[0] = u;
  mc.nin = 1;
  mc.out[0] = d_out;
  mc.nout = 1;
  return run_map(ctx, tets, mc, OP_DIAG, opts);
}

// Spring-mass system (Section 4.1, Figure 1) on the edge relation.
namespace {
ebb_status_t springs_checks(ebb_ctx_t ctx, ebb_rel_t tets) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (!tets) return set_error(ctx, EBB_ERR_ARG, "null relation");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  if (tets->edges.row_off == nullptr)
    return set_error(ctx, EBB_ERR_STATE, "relation finalized without EBB_FINALIZE_EDGES");
  if (tets->vperm) return set_error(ctx, EBB_ERR_STATE, "springs do not support EBB_FINALIZE_REORDER_VERTS");
  return EBB_OK;
}
}  // namespace

ebb_status_t ebb_springs_init(ebb_ctx_t ctx, ebb_rel_t tets, const char* pos) {
  ebb_status_t s = springs_checks(ctx, tets);
  if (s) return s;
  const Field* f = pos ? find_field(tets->verts, pos) : nullptr;
  if (!f || f->ncomp != 3 || (f->dtype != EBB_F64 && f->dtype != EBB_F32))
    return set_error(ctx, EBB_ERR_ARG, "pos must name an F64 or F32 vertex field with 3 components");
  cudaError_t e = springs_init(tets, f->ptr, f->dtype == EBB_F64, ctx->stream);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, "device allocation for the springs failed");
  }
  return cuda_check(ctx, e, "spring rest lengths");
}

ebb_status_t ebb_springs_run(ebb_ctx_t ctx, ebb_rel_t tets, const char* q, const char* qd, const char* mass,
                             double k, double dt, int32_t steps, double* energy) {
  ebb_status_t s = springs_checks(ctx, tets);
  if (s) return s;
  if (!tets->edges.springs_ready) return set_error(ctx, EBB_ERR_STATE, "call ebb_springs_init first");
  if (steps < 0 || !(dt >= 0.0) || !std::isfinite(k)) return set_error(ctx, EBB_ERR_ARG, "need steps >= 0, dt >= 0");
  const Field* fq = q ? find_field(tets->verts, q) : nullptr;
  if (!fq || fq->ncomp != 3 || (fq->dtype != EBB_F64 && fq->dtype != EBB_F32))
    return set_error(ctx, EBB_ERR_ARG, "q must name an F64 or F32 vertex field with 3 components");
  void *pqd = nullptr, *pm = nullptr;
  s = vertex_field(ctx, tets, qd, fq->dtype, 3, &pqd);
  if (!s) s = vertex_field(ctx, tets, mass, fq->dtype, 1, &pm);
  if (s) return s;
  const size_t es = fq->dtype == EBB_F64 ? 8 : 4;
  const size_t nv = (size_t)tets->verts->size;
  if (ranges_overlap(fq->ptr, 3 * nv * es, pqd, 3 * nv * es) || ranges_overlap(fq->ptr, 3 * nv * es, pm, nv * es) ||
      ranges_overlap(pqd, 3 * nv * es, pm, nv * es))
    return set_error(ctx, EBB_ERR_PHASE, "q, qd and mass must be three distinct fields");
  cudaError_t e = springs_run(tets, fq->ptr, pqd, pm, fq->dtype == EBB_F64, k, dt, steps, energy, ctx->stream);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, "device allocation for the springs failed");
  }
  return cuda_check(ctx, e, "spring steps");
}

ebb_status_t ebb_assemble_tet_K(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const ebb_map_opts_t* opts) {
  if (ctx && tets && tets->ctx == ctx && tets->finalized && tets->edges.row_off == nullptr)
    return set_error(ctx, EBB_ERR_STATE, "relation finalized without EBB_FINALIZE_EDGES");
  MapCall mc;
  mc.in[0] = u;
  mc.nin = 1;
  mc.nout = 0;
  return run_map(ctx, tets, mc, OP_ASSEMBLE, opts);
}

ebb_status_t ebb_spmv_tet_K(ebb_ctx_t ctx, ebb_rel_t tets, const char* w, const char* Kw_out,
                            const ebb_map_opts_t* opts) {
  if (ctx && tets && opts && tets->ctx == ctx && tets->finalized) {
    if (tets->edges.row_off == nullptr)
      return set_error(ctx, EBB_ERR_STATE, "relation finalized without EBB_FINALIZE_EDGES");
    if (!tets->edges.assembled[opts->precision == EBB_PREC_F64 ? 1 : 0])
      return set_error(ctx, EBB_ERR_STATE, "no stiffness assembled in this precision (call ebb_assemble_tet_K)");
  }
  MapCall mc;
  mc.in[0] = w;
  mc.nin = 1;
  mc.out[0] = Kw_out;
  mc.nout = 1;
  return run_map(ctx, tets, mc, OP_SPMV, opts);
}

ebb_status_t ebb_relation_set_tuning(ebb_ctx_t ctx, ebb_rel_t tets, int32_t model, int32_t precision,
                                     int32_t reduce, int32_t tile_tets, int32_t flags) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (!tets) return set_error(ctx, EBB_ERR_ARG, "null relation");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  if ((model != EBB_STVK && model != EBB_NEOHOOKEAN) || (precision != EBB_PREC_F64 && precision != EBB_PREC_F32) ||
      !valid_reduce(reduce) || tile_tets < 1 ||
      tile_tets > kTileTets || (flags & ~(int32_t)(EBB_TUNE_INTERLEAVED | EBB_TUNE_RECORD_PLANES)) != 0)
    return set_error(ctx, EBB_ERR_ARG, "tuning value out of range");
  if (reduce == EBB_REDUCE_COLOR && !tets->has_colour)
    return set_error(ctx, EBB_ERR_STATE, "colour reduction requested but relation finalized without EBB_FINALIZE_COLOR");
  if (tets->tile_cap != tile_tets) {
    ebb_status_t s = retile(ctx, tets, tile_tets);
    if (s) return s;
  }
  tets->tuned[model][precision] = (signed char)reduce;
  tets->stage_interleaved = (flags & EBB_TUNE_INTERLEAVED) != 0;
  const bool planes = (flags & EBB_TUNE_RECORD_PLANES) != 0;
  if (planes != tets->rec_planes) {
    ebb_status_t s = repack_records(ctx, tets, planes);
    if (s) return s;
  }
  return EBB_OK;
}

ebb_status_t ebb_relation_autotune(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* w,
                                   const ebb_map_opts_t* opts, ebb_autotune_report_t* report) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (report) memset(report, 0, sizeof *report);
  if (!tets || !opts || !u || !w || !report) return set_error(ctx, EBB_ERR_ARG, "null argument");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  if (opts->model != EBB_STVK && opts->model != EBB_NEOHOOKEAN)
    return set_error(ctx, EBB_ERR_ARG, "unknown material model");
  if (opts->precision != EBB_PREC_F64 && opts->precision != EBB_PREC_F32)
    return set_error(ctx, EBB_ERR_ARG, "unknown precision");
  const bool f64 = opts->precision == EBB_PREC_F64;
  void* in[2] = {nullptr, nullptr};
  bool x4 = false;
  const char* names[2] = {u, w};
  ebb_status_t s = map_fields(ctx, tets, names, 2, f64, in, &x4);
  if (s) return s;
  s = read_device_error(ctx);
  if (s) return s;
  const int nv = (int)tets->verts->size;
  const size_t bytes = (size_t)nv * (x4 ? 16 : 3 * (f64 ? 8 : 4));
  cudaStream_t st = ctx->stream;
  void* out[1] = {nullptr};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaMalloc(&out[0], bytes > 0 ? bytes : 16);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  auto cleanup = [&]() {
    cudaFree(out[0]);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (ce != cudaSuccess) {
    cleanup();
    cudaGetLastError();
    return set_error(ctx, EBB_ERR_NOMEM, "autotune scratch allocation failed");
  }
  // Time one candidate as a map call runs it (staging included): median of 7
  // launches after 2 untimed ones.
  auto time_map = [&](ebb_reduce_t reduce, double* us) -> ebb_status_t {
    std::vector<float> t;
    for (int it = 0; it < 9; ++it) {
      cudaError_t e = cudaMemsetAsync(out[0], 0, bytes, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e != cudaSuccess) return cuda_check(ctx, e, "autotune timing");
      ebb_status_t ms = launch_map_staged(ctx, tets, OP_KV, opts->model, opts->mu, opts->lambda, reduce, f64, x4, in,
                                          2, out, 1, false);
      if (ms) return ms;
      e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float msec = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&msec, e0, e1);
      if (e != cudaSuccess) return cuda_check(ctx, e, "autotune timing");
      if (it >= 2) t.push_back(msec);
    }
    std::sort(t.begin(), t.end());
    *us = 1e3 * t[t.size() / 2];
    return EBB_OK;
  };
  int nc = 0;
  double best_tiled_us = 1e300, best_us = 1e300;
  int best_cap = tets->tile_cap;
  ebb_reduce_t best = EBB_REDUCE_TILED;
  tets->stage_interleaved = false;
  if (tets->rec_planes) s = repack_records(ctx, tets, false);   // tile sizes are timed with row records
  const int caps[3] = {128, 96, 64};
  for (int ci = 0; ci < 3 && !s; ++ci) {
    if (tets->tile_cap != caps[ci]) {
      s = retile(ctx, tets, caps[ci]);
      if (s) break;
    }
    double us = 0.0;
    s = time_map(EBB_REDUCE_TILED, &us);
    if (s) break;
    report->cand[nc++] = ebb_autotune_cand_t{EBB_REDUCE_TILED, caps[ci], x4 ? 1 : 0, tets->rec_planes ? 1 : 0, us};
    if (us < best_tiled_us) {
      best_tiled_us = us;
      best_cap = caps[ci];
    }
  }
  if (!s && tets->tile_cap != best_cap) s = retile(ctx, tets, best_cap);
  if (!s && !f64 && !x4) {
    // the same tile size with the operands staged vertex-interleaved
    tets->stage_interleaved = true;
    double us = 0.0;
    s = time_map(EBB_REDUCE_TILED, &us);
    if (!s) {
      report->cand[nc++] = ebb_autotune_cand_t{EBB_REDUCE_TILED, best_cap, 1, tets->rec_planes ? 1 : 0, us};
      if (us < best_tiled_us) best_tiled_us = us;
      else tets->stage_interleaved = false;
    }
  }
  if (!s) {
    // the same configuration with the other record layout
    const bool was = tets->rec_planes;
    s = repack_records(ctx, tets, !was);
    double us = 0.0;
    if (!s) s = time_map(EBB_REDUCE_TILED, &us);
    if (!s) {
      report->cand[nc++] = ebb_autotune_cand_t{EBB_REDUCE_TILED, best_cap,
                                               (!f64 && (x4 || tets->stage_interleaved)) ? 1 : 0, !was ? 1 : 0, us};
      if (us < best_tiled_us)
        best_tiled_us = us;
      else
        s = repack_records(ctx, tets, was);
    }
  }
  const ebb_reduce_t others[4] = {EBB_REDUCE_ATOMIC, EBB_REDUCE_GATHER, EBB_REDUCE_COOP, EBB_REDUCE_COLOR};
  for (int oi = 0; oi < 4 && !s; ++oi) {
    if (others[oi] == EBB_REDUCE_COLOR && !tets->has_colour) continue;
    double us = 0.0;
    s = time_map(others[oi], &us);
    if (s) break;
    report->cand[nc++] = ebb_autotune_cand_t{others[oi], 0, x4 ? 1 : 0, 0, us};
    if (us < best_us) {
      best_us = us;
      best = others[oi];
    }
  }
  cleanup();
  if (s) return s;
  s = read_device_error(ctx);
  if (s) return s;
  if (best_tiled_us <= best_us) best = EBB_REDUCE_TILED;
  tets->tuned[opts->model][opts->precision] = (signed char)best;
  report->reduce = best;
  report->tile_tets = tets->tile_cap;
  report->interleaved = (!f64 && (x4 || tets->stage_interleaved)) ? 1 : 0;
  report->record_planes = tets->rec_planes ? 1 : 0;
  report->ncand = nc;
  return EBB_OK;
}

ebb_status_t ebb_relation_info(ebb_ctx_t ctx, ebb_rel_t tets, ebb_relation_info_t* info) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (!tets || !info) return set_error(ctx, EBB_ERR_ARG, "null argument");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  memset(info, 0, sizeof *info);
  info->n_tets = tets->size;
  info->n_verts = tets->verts->size;
  info->ntiles = tets->tiles.ntiles;
  info->tile_tets = tets->tile_cap;
  info->ncolours = tets->has_colour ? tets->colour.ncolours : 0;
  info->interleaved = tets->stage_interleaved ? 1 : 0;
  info->reordered = tets->vperm != nullptr ? 1 : (tets->vorder.empty() ? 0 : 2);
  info->record_planes = tets->rec_planes ? 1 : 0;
  for (int m = 0; m < 2; ++m)
    for (int p = 0; p < 2; ++p) info->tuned[m][p] = tets->tuned[m][p];
  return EBB_OK;
}

ebb_status_t ebb_relation_vertex_order(ebb_ctx_t ctx, ebb_rel_t tets, int32_t* order, int64_t n) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (!tets) return set_error(ctx, EBB_ERR_ARG, "null relation");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  const int64_t nv = tets->verts->size;
  if (n != nv || (nv > 0 && !order)) return set_error(ctx, EBB_ERR_ARG, "order needs exactly one entry per vertex");
  for (int64_t i = 0; i < nv; ++i) order[i] = tets->vorder.empty() ? (int32_t)i : tets->vorder[i];
  return EBB_OK;
}

ebb_status_t ebb_cg_implicit_step(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* v, const char* pinned,
                                  const ebb_step_params_t* params, ebb_cg_report_t* report) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (report) {
    report->iters = 0;
    report->rel_residual = 0.0;
    report->status = EBB_ERR_ARG;
  }
  if (!tets || !params || !u || !v) return set_error(ctx, EBB_ERR_ARG, "null argument");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  if (params->model != EBB_STVK && params->model != EBB_NEOHOOKEAN)
    return set_error(ctx, EBB_ERR_ARG, "unknown material model");
  if (params->precision != EBB_PREC_F64 && params->precision != EBB_PREC_F32)
    return set_error(ctx, EBB_ERR_ARG, "unknown precision");
  if (!(params->dt > 0.0) || !(params->rho > 0.0) || params->max_iters < 0 || !(params->rtol >= 0.0))
    return set_error(ctx, EBB_ERR_ARG, "need dt > 0, rho > 0, max_iters >= 0, rtol >= 0");
  ebb_reduce_t reduce = resolve_reduce(tets, params->reduce, params->model, params->precision);
  if (!valid_reduce(reduce))
    return set_error(ctx, EBB_ERR_ARG, "unknown reduction variant");
  if (reduce == EBB_REDUCE_COLOR && !tets->has_colour)
    return set_error(ctx, EBB_ERR_STATE, "colour reduction requested but relation finalized without EBB_FINALIZE_COLOR");
  if (params->flags & ~EBB_STEP_ASSEMBLED) return set_error(ctx, EBB_ERR_ARG, "unknown EBB_STEP_* flag");
  if ((params->flags & EBB_STEP_ASSEMBLED) && tets->edges.row_off == nullptr)
    return set_error(ctx, EBB_ERR_STATE, "EBB_STEP_ASSEMBLED needs a relation finalized with EBB_FINALIZE_EDGES");
  void *pu = nullptr, *pv = nullptr;
  ebb_status_t s = vertex_field(ctx, tets, u, EBB_F64, 3, &pu);
  if (s) return s;
  s = vertex_field(ctx, tets, v, EBB_F64, 3, &pv);
  if (s) return s;
  const size_t bytes = (size_t)tets->verts->size * 3 * 8;
  if (ranges_overlap(pu, bytes, pv, bytes))
    return set_error(ctx, EBB_ERR_PHASE, "u and v overlap");
  const void* pp = nullptr;
  ebb_dtype_t pdt = EBB_U8;
  if (pinned) {
    const Field* f = find_field(tets->verts, pinned);
    if (!f || f->ncomp != 1 || (f->dtype != EBB_U8 && f->dtype != EBB_I32))
      return set_error(ctx, EBB_ERR_ARG, "pinned must name a U8 or I32 vertex field with 1 component");
    pp = f->ptr;
    pdt = f->dtype;
  }
  ebb_step_params_t p = *params;
  p.reduce = reduce;
  return run_implicit_step(ctx, tets, (double*)pu, (double*)pv, pp, pdt, &p, report);
}

namespace {
ebb_status_t step_vjp_entry(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* v, const char* v_next,
                            const char* pinned, const char* gu, const char* gv, const char* gmu, const char* glam,
                            const ebb_step_params_t* params, ebb_cg_report_t* report) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (report) *report = ebb_cg_report_t{0, 0.0, EBB_ERR_ARG};
  if (!tets || !params || !u || !v || !gu || !gv) return set_error(ctx, EBB_ERR_ARG, "null argument");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  if (params->model != EBB_STVK || params->precision != EBB_PREC_F64)
    return set_error(ctx, EBB_ERR_ARG, "the step VJP supports StVK in FP64 only");
  if (params->flags != 0) return set_error(ctx, EBB_ERR_ARG, "the step VJP takes no EBB_STEP_* flags");
  if (tets->vperm) return set_error(ctx, EBB_ERR_STATE, "the step VJP does not support EBB_FINALIZE_REORDER_VERTS");
  if (!(params->dt > 0.0) || !(params->rho > 0.0) || params->max_iters < 0 || !(params->rtol >= 0.0))
    return set_error(ctx, EBB_ERR_ARG, "need dt > 0, rho > 0, max_iters >= 0, rtol >= 0");
  ebb_reduce_t reduce = resolve_reduce(tets, params->reduce, params->model, params->precision);
  if (!valid_reduce(reduce))
    return set_error(ctx, EBB_ERR_ARG, "unknown reduction variant");
  if (reduce == EBB_REDUCE_COLOR && !tets->has_colour)
    return set_error(ctx, EBB_ERR_STATE, "colour reduction requested but relation finalized without EBB_FINALIZE_COLOR");
  void *pu = nullptr, *pv = nullptr, *pgu = nullptr, *pgv = nullptr, *pvn = nullptr;
  ebb_status_t s = vertex_field(ctx, tets, u, EBB_F64, 3, &pu);
  if (!s) s = vertex_field(ctx, tets, v, EBB_F64, 3, &pv);
  if (!s) s = vertex_field(ctx, tets, gu, EBB_F64, 3, &pgu);
  if (!s) s = vertex_field(ctx, tets, gv, EBB_F64, 3, &pgv);
  if (!s && v_next) s = vertex_field(ctx, tets, v_next, EBB_F64, 3, &pvn);
  if (s) return s;
  const size_t bytes = (size_t)tets->verts->size * 3 * 8;
  const void* all[5] = {pu, pv, pgu, pgv, pvn};
  const int nall = pvn ? 5 : 4;
  for (int i = 0; i < nall; ++i)
    for (int j = i + 1; j < nall; ++j)
      if (ranges_overlap(all[i], bytes, all[j], bytes))
        return set_error(ctx, EBB_ERR_PHASE, "u, v, v_next, gu and gv must be distinct fields");
  double* per_tet[2] = {nullptr, nullptr};
  const char* names[2] = {gmu, glam};
  for (int i = 0; i < 2; ++i) {
    if (!names[i]) continue;
    const Field* f = find_field(tets, names[i]);
    if (!f || f->dtype != EBB_F64 || f->ncomp != 1)
      return set_error(ctx, EBB_ERR_ARG, std::string("per-tet gradient field '") + names[i] +
                                             "' must be bound on tets as F64 with 1 component");
    per_tet[i] = (double*)f->ptr;
  }
  const void* pp = nullptr;
  ebb_dtype_t pdt = EBB_U8;
  if (pinned) {
    const Field* f = find_field(tets->verts, pinned);
    if (!f || f->ncomp != 1 || (f->dtype != EBB_U8 && f->dtype != EBB_I32))
      return set_error(ctx, EBB_ERR_ARG, "pinned must name a U8 or I32 vertex field with 1 component");
    pp = f->ptr;
    pdt = f->dtype;
  }
  ebb_step_params_t p = *params;
  p.reduce = reduce;
  return run_step_vjp(ctx, tets, (const double*)pu, (const double*)pv, (const double*)pvn, pp, pdt, (double*)pgu,
                      (double*)pgv, per_tet[0], per_tet[1], &p, report);
}
}  // namespace

ebb_status_t ebb_cg_implicit_step_vjp(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* v,
                                      const char* pinned, const char* gu, const char* gv, const char* gmu,
                                      const char* glam, const ebb_step_params_t* params, ebb_cg_report_t* report) {
  return step_vjp_entry(ctx, tets, u, v, nullptr, pinned, gu, gv, gmu, glam, params, report);
}

ebb_status_t ebb_cg_implicit_step_vjp_at(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* v,
                                         const char* v_next, const char* pinned, const char* gu, const char* gv,
                                         const char* gmu, const char* glam, const ebb_step_params_t* params,
                                         ebb_cg_report_t* report) {
  if (!v_next) {
    if (ctx) return set_error(ctx, EBB_ERR_ARG, "null v_next");
    return EBB_ERR_ARG;
  }
  return step_vjp_entry(ctx, tets, u, v, v_next, pinned, gu, gv, gmu, glam, params, report);
}

ebb_status_t ebb_cg_implicit_step_batched(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const char* v,
                                          const char* pinned, const char* batch, int32_t nbatch,
                                          const ebb_step_params_t* params, ebb_cg_report_t* reports) {
  if (!ctx) return EBB_ERR_ARG;
  ctx->last_error.clear();
  if (reports)
    for (int32_t m = 0; m < nbatch; ++m) reports[m] = ebb_cg_report_t{0, 0.0, EBB_ERR_ARG};
  if (!tets || !params || !u || !v || !batch || nbatch < 1) return set_error(ctx, EBB_ERR_ARG, "null argument");
  if (tets->ctx != ctx) return set_error(ctx, EBB_ERR_ARG, "relation belongs to another context");
  if (!tets->finalized) return set_error(ctx, EBB_ERR_STATE, "relation not finalized");
  if (params->model != EBB_STVK && params->model != EBB_NEOHOOKEAN)
    return set_error(ctx, EBB_ERR_ARG, "unknown material model");
  if (params->precision != EBB_PREC_F64 && params->precision != EBB_PREC_F32)
    return set_error(ctx, EBB_ERR_ARG, "unknown precision");
  if (!(params->dt > 0.0) || !(params->rho > 0.0) || params->max_iters < 0 || !(params->rtol >= 0.0))
    return set_error(ctx, EBB_ERR_ARG, "need dt > 0, rho > 0, max_iters >= 0, rtol >= 0");
  ebb_reduce_t reduce = resolve_reduce(tets, params->reduce, params->model, params->precision);
  if (!valid_reduce(reduce))
    return set_error(ctx, EBB_ERR_ARG, "unknown reduction variant");
  if (reduce == EBB_REDUCE_COLOR && !tets->has_colour)
    return set_error(ctx, EBB_ERR_STATE, "colour reduction requested but relation finalized without EBB_FINALIZE_COLOR");
  if (tets->verts->size == 0) return set_error(ctx, EBB_ERR_ARG, "empty vertex relation");
  if (tets->vperm) return set_error(ctx, EBB_ERR_STATE, "the batched step does not support EBB_FINALIZE_REORDER_VERTS");
  if (params->flags != 0) return set_error(ctx, EBB_ERR_ARG, "the batched step takes no EBB_STEP_* flags");
  void *pu = nullptr, *pv = nullptr, *pb = nullptr;
  ebb_status_t s = vertex_field(ctx, tets, u, EBB_F64, 3, &pu);
  if (s) return s;
  s = vertex_field(ctx, tets, v, EBB_F64, 3, &pv);
  if (s) return s;
  s = vertex_field(ctx, tets, batch, EBB_I32, 1, &pb);
  if (s) return s;
  const size_t bytes = (size_t)tets->verts->size * 3 * 8;
  if (ranges_overlap(pu, bytes, pv, bytes)) return set_error(ctx, EBB_ERR_PHASE, "u and v overlap");
  const void* pp = nullptr;
  if (pinned) {
    const Field* f = find_field(tets->verts, pinned);
    if (!f || f->ncomp != 1 || f->dtype != EBB_U8)
      return set_error(ctx, EBB_ERR_ARG, "pinned must name a U8 vertex field with 1 component");
    pp = f->ptr;
  }
  ebb_step_params_t p = *params;
  p.reduce = reduce;
  return run_batched_step(ctx, tets, (double*)pu, (double*)pv, pp, (const int*)pb, nbatch, &p, reports);
}

}  // extern "C"
