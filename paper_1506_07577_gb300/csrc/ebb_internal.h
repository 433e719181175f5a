// Internal structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/ebb.h"

namespace ebb {

// Device status word: [0] = first error code, [1] = row index it refers to.
enum { ERRW_CODE = 0, ERRW_INDEX = 1, ERRW_WORDS = 4 };

struct Field {
  std::string name;
  ebb_dtype_t dtype = EBB_F64;
  int ncomp = 1;
  void* ptr = nullptr;
  ebb_rel_s* key_target = nullptr;
};

// Per-tet streams in the layout the kernels read.  Matrices are 9 planes of
// nt elements (entry (r,c) of B at B[(3r+c)*nt + t]).
template <typename T>
struct TetStreams {
  T* B = nullptr;
  T* V = nullptr;
  T* mu = nullptr;   // null: uniform material
  T* lam = nullptr;
};

// Vertex-conflict colouring of the tets: tets of colour c are the internal
// rows [offsets[c], offsets[c+1]) of the colour-ordered copy.
struct Colouring {
  int ncolours = 0;
  std::vector<int> offsets;
  int4* keys = nullptr;
  TetStreams<double> s64;
  TetStreams<float> s32;
};

struct StepScratch;  // defined in cg.cu

struct ebb_rel_impl;

}  // namespace ebb

struct ebb_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string last_error;
  int* d_err = nullptr;     // device status word (ERRW_WORDS ints)
  int* h_err = nullptr;     // pinned host mirror
  std::vector<ebb_rel_s*> rels;
};

struct ebb_rel_s {
  ebb_ctx_s* ctx = nullptr;
  std::string name;
  int64_t size = 0;
  std::map<std::string, ebb::Field> fields;

  // ---- finalized tet data (tets relation only) ----
  bool finalized = false;
  ebb_rel_s* verts = nullptr;
  int4* keys = nullptr;                 // internal keys, one int4 per tet
  ebb::TetStreams<double> s64;
  ebb::TetStreams<float> s32;
  ebb::Colouring colour;
  bool has_colour = false;

  // ---- implicit-step scratch ----
  ebb::StepScratch* step = nullptr;
};

namespace ebb {

// error helpers (abi.cu)
ebb_status_t set_error(ebb_ctx_s* ctx, ebb_status_t code, const std::string& msg);
ebb_status_t cuda_check(ebb_ctx_s* ctx, cudaError_t e, const char* what);

// Element map launch (tet_maps.cu).
enum MapOps { OP_FORCE = 1, OP_KV = 2, OP_DIAG = 4 };

template <typename T>
struct MapIO {
  const T* u = nullptr;    // displacement, 3 planes of nv
  const T* w = nullptr;    // direction for K w
  T* f = nullptr;          // force accumulator
  T* Kw = nullptr;         // K w accumulator
  T* d = nullptr;          // diag(K) accumulator
};

// Launch one element map over all tets of `rel` on `stream`.  `active`
// (device int, may be null) lets the kernel return early when *active == 0
// (CG iterations after convergence).
template <typename T>
cudaError_t launch_tet_map(ebb_rel_s* rel, int model, int ops, ebb_reduce_t reduce,
                           T mu0, T lam0, const MapIO<T>& io, const int* active,
                           cudaStream_t stream);

// Free the per-relation step scratch (cg.cu).
void free_step_scratch(ebb_rel_s* rel);

// Run one implicit step (cg.cu).
ebb_status_t run_implicit_step(ebb_ctx_s* ctx, ebb_rel_s* tets, double* u, double* v,
                               const void* pinned, ebb_dtype_t pinned_dtype,
                               const ebb_step_params_t* p, ebb_cg_report_t* rep);

// Build the colouring (colour.cu).
ebb_status_t build_colouring(ebb_ctx_s* ctx, ebb_rel_s* tets);
void free_colouring(ebb_rel_s* tets);

}  // namespace ebb
