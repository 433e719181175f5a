// Internal structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/ebb.h"
#include "host_parallel.h"

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
  int* perm = nullptr;   // colour-ordered row -> caller's row
  TetStreams<double> s64;
  TetStreams<float> s32;
};

// Tiles of consecutive (Morton-ordered) tets for the shared-memory maps.
// A tile holds up to kTileTets tets touching at most kTileSlots distinct
// vertices ("slots").  Everything a tile needs except the vertex fields is
// packed into one contiguous blob:
//   header  int4 {ntets, nslots, first internal tet row, nunits}
//   slots   uchar4[kTileTets]        tile-local slot of each tet corner
//   ent     u16[kTileTets][kUnitEntries]  entries summed by thread i: entry
//                                    (corner a, tet t) is coded as the row
//                                    3a*(kTileTets+1) + t of the per-corner
//                                    output array (rows 3a+c of kTileTets+1
//                                    columns); an unused step holds
//                                    kEntryNone.  The steps are ordered so
//                                    that the 16 threads of a half-warp hit
//                                    distinct bank pairs where possible
//   units   u32[kTileTets]           reduction work of thread i: bit 0 has a
//                                    unit, 14-21 slot, 22-25 lanes after this
//                                    one in the same slot and warp, 26 first
//                                    lane of that run (adds the sum into the
//                                    field)
//   vtx     int[kTileSlots]          vertex id of each slot
//   rec     the per-tet element data in one of two layouts (a tuning
//           choice, BlobLayout::planes):
//           rows    T[kTileTets][rec_len<T>] one row-oriented record per tet
//                   (the fields one element uses together): Dm^-1 entries
//                   (r,c) at 3r+c, rest volume at 9, Lame mu, lambda at 10,
//                   11 (zero without per-tet material), then padding; 48 B
//                   (FP32) or 112 B (FP64), strides at which a thread's
//                   16-byte loads stay free of bank conflicts
//           planes  T[12][kTileTets] one plane per field (Dm^-1 entries,
//                   V, mu, lambda): consecutive tets' values adjacent; without
//                   per-tet material the last two planes are not copied
// Unused tail entries are zero.
constexpr int kTileTets = 128;   // tets per tile (= threads per CTA)
constexpr int kTileSlots = 128;  // distinct vertices per tile (u8 slots)
constexpr int kUnitEntries = 8;  // entries summed by one thread
constexpr int kUnitMaxRun = 16;  // units of one slot (4-bit lane count)
constexpr unsigned short kEntryNone = 0xffff;
constexpr int kBlobSlots = 16;
constexpr int kBlobEnt = kBlobSlots + 4 * kTileTets;
constexpr int kBlobUnits = kBlobEnt + 2 * kUnitEntries * kTileTets;
constexpr int kBlobVtx = kBlobUnits + 4 * kTileTets;
constexpr int kBlobPrefix = kBlobVtx + 4 * kTileSlots;
static_assert(kBlobPrefix % 16 == 0, "blob prefix must keep 16-byte alignment");
static_assert(kTileTets < 256 && kTileSlots <= 256, "entry code and unit descriptor field widths");

// Per-tet record length of the tile blobs, in elements.
template <typename T>
constexpr int rec_len() {
  return sizeof(T) == 4 ? 12 : 14;
}

struct BlobLayout {
  int bytes = 0;           // per tile (multiple of 128)
  int copy = 0;            // bytes a kernel copies per tile (multiple of 16, <= bytes)
  int rec = 0;             // byte offset of the per-tet records
  bool material = false;   // records carry per-tet Lame parameters
  bool planes = false;     // per-tet data as field planes instead of row records
};

// Partial-row index of the ordered tiled variant (EBB_REDUCE_TILED_ORDERED).
// The rows are numbered vertex by vertex: the vertices that own rows are
// listed in order of first use by the tiles (ord_vtx, n_ord of them), and
// vertex ord_vtx[i] owns rows ord_off[i] .. ord_off[i+1], one per tile whose
// units add into it, in tile order.  unit_row[t * kTileTets + i] is the row
// of reduction unit i of tile t when that unit heads a vertex's run (-1
// otherwise); the tile pass reads it at the start of the tile, so that the
// second pass reads every vertex's rows contiguously.
struct Tiles {
  int ntiles = 0;
  unsigned char* blob32 = nullptr;
  unsigned char* blob64 = nullptr;
  BlobLayout L32, L64;
  int n_ord = 0;
  int* ord_off = nullptr;
  int* ord_vtx = nullptr;
  int* unit_row = nullptr;
  // Partial rows (ntiles * kTileTets rows of 3 fields x 4 values), [0] FP32,
  // [1] FP64; allocated at first use.
  void* partial[2] = {nullptr, nullptr};
};

// Inverse of the key-field (Section 6.1 GroupBy): for vertex v the entries
// ent[off[v] .. off[v+1]) are 4*t + a for every internal tet row t whose
// corner a is v, in increasing order.
// `order` lists the vertices by their first entry (the vertices of tet 0
// first, ...): a per-vertex pass walked in this order reads the per-corner
// data of nearby tets together, whatever the vertex numbering.
struct VertexIndex {
  int* off = nullptr;
  int* ent = nullptr;
  int* order = nullptr;
};

// Edge relation with self-loops (Section 5.2) as block CSR over internal
// vertices: row r's blocks are (r, col[k]), k in [row_off[r], row_off[r+1]),
// columns increasing; tet_blk[16 t + 4 a + b] is the block of corners (a, b)
// of internal tet t (the key-field tets.e[4][4]).  blocks[p]: the assembled
// stiffness as 9 planes of nnzb, entry (c, d) of block k at [(3 c + d) nnzb
// + k] ([0] FP32, [1] FP64).
struct EdgeIndex {
  int nnzb = 0;
  int* row_off = nullptr;
  int* col = nullptr;
  int* tet_blk = nullptr;
  void* blocks[2] = {nullptr, nullptr};
  bool assembled[2] = {false, false};
  // Spring-mass system on the edges: rest length per entry (the self-loop's
  // unused), double-buffered positions, energy partial sums.
  void* rest[2] = {nullptr, nullptr};
  void* qbuf[2] = {nullptr, nullptr};
  double* epart = nullptr;
  bool springs_ready = false;
};

struct StepScratch;   // defined in cg.cu

// Chunk plan of the host-buffer map (abi.cu): the tiles cut into K
// consecutive ranges.  Before chunk c runs, the input rows [0, need_hi[c])
// are on the device; after it, the output rows [0, done_lo[c]) are final (no
// later chunk adds to them).  On a relation whose vertices are numbered in
// Morton order consecutive tiles touch nearly consecutive rows, so the
// copies of one chunk overlap the map of another.
struct HostPlan {
  static constexpr int kChunks = 6;
  unsigned gen = ~0u;
  int K = 0;
  std::vector<int> tile_off, need_hi, done_lo;
  int own = 0;      // rows [own, nv): shared by several chunks (copied in first, out last)
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  cudaEvent_t ev_in[kChunks] = {}, ev_map[kChunks] = {};
};
// First tile of chunk c of K consecutive chunks over ntiles tiles (c = K:
// ntiles).  With K = HostPlan::kChunks the chunks hold 1, 3, 4, 4, 3 and 1
// sixteenths of the tiles: the first and last are small, so that the copy-in
// before the first map and the copy-out after the last are short, and the
// others large, so that few launches pay a map's ramp and tail.  Other
// counts cut evenly.
inline int chunk_first_tile(int c, int ntiles, int K) {
  static const int kEnd[HostPlan::kChunks + 1] = {0, 1, 4, 8, 12, 15, 16};
  static_assert(HostPlan::kChunks == 6, "chunk weights");
  if (K != HostPlan::kChunks) return (int)((long long)c * ntiles / K);
  return (int)((long long)kEnd[c] * ntiles / kEnd[HostPlan::kChunks]);
}

struct BatchScratch;  // defined in batched.cu

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
  int4* keys = nullptr;                 // internal keys, one int4 per tet (Morton order)
  int* tet_perm = nullptr;              // internal row -> caller's row
  int* vperm = nullptr;                 // internal vertex -> caller's vertex (null: same order)
  std::vector<int> vorder;              // EBB_FINALIZE_RENUMBER_VERTS: row i was the caller's vertex vorder[i]
  int vown = -1;                        // rows before the vertices several host-map chunks share (-1: none)
  void* vscratch[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // reordered map operands
  ebb::TetStreams<double> s64;
  ebb::TetStreams<float> s32;
  ebb::Colouring colour;
  bool has_colour = false;
  ebb::Tiles tiles;
  int tile_cap = ebb::kTileTets;        // tets per tile the layout was cut with
  unsigned layout_gen = 0;              // bumped whenever the tile blobs are rebuilt
  signed char tuned[2][2] = {{-1, -1}, {-1, -1}};  // autotuned reduce per [model][precision], -1 none
  int test_drop_tile = -1;              // EBB_MAP_TEST_DROP_TILE: tile whose blob copy the next map skips
  bool stage_interleaved = false;       // FP32 tiled maps stage operands vertex-interleaved (autotuned)
  bool rec_planes = false;              // tile blobs hold per-tet data as planes (autotuned)
  ebb::VertexIndex vindex;
  void* gather_corner[2] = {nullptr, nullptr};  // EBB_REDUCE_GATHER per-corner buffers, [0] FP32, [1] FP64
  ebb::EdgeIndex edges;                 // built with EBB_FINALIZE_EDGES

  // ---- implicit-step scratch ----
  ebb::StepScratch* step = nullptr;
  ebb::HostPlan* hplan = nullptr;       // chunk plan of the host-buffer map (abi.cu)
  float* xyz_stage = nullptr;           // host-buffer map's packed-row staging: u, w, f, Kw, 3 x N_v floats
                                        // each (EBB_MAP_HOST_XYZ; allocated on first use)
  ebb::BatchScratch* batch = nullptr;
};

namespace ebb {

// error helpers (abi.cu)
ebb_status_t set_error(ebb_ctx_s* ctx, ebb_status_t code, const std::string& msg);
ebb_status_t cuda_check(ebb_ctx_s* ctx, cudaError_t e, const char* what);

// Element map launch (tet_maps.cu).
enum MapOps { OP_FORCE = 1, OP_KV = 2, OP_DIAG = 4, OP_ASSEMBLE = 8, OP_SPMV = 16 };

template <typename T>
struct MapIO {
  const T* u = nullptr;    // displacement, 3 planes of nv
  const T* w = nullptr;    // direction for K w
  T* f = nullptr;          // force accumulator
  T* Kw = nullptr;         // K w accumulator
  T* d = nullptr;          // diag(K) accumulator
  // Ordered tiled reduction only: each run total is stored to its partial
  // row (NF groups of 4 values: x, y, z, 0; row index from unit_row) instead
  // of added to the fields.
  T* part = nullptr;
  const int* unit_row = nullptr;
  // Tiled (unordered) reduction: map only the tiles [tile_begin, tile_end)
  // (tile_end < 0: to the last tile).
  int tile_begin = 0;
  int tile_end = -1;
  // Vertex-interleaved operands (library-internal fields only): every field
  // above is nv groups of 4 (x, y, z, padding) instead of 3 planes; FP32 and
  // the tiled reduction only.
  bool aos = false;
};

// Launch one element map over all tets of `rel` on `stream`.  `active`
// (device int, may be null) lets the kernel return early when *active == 0
// (CG iterations after convergence).
template <typename T>
cudaError_t launch_tet_map(ebb_rel_s* rel, int model, int ops, ebb_reduce_t reduce,
                           T mu0, T lam0, const MapIO<T>& io, const int* active,
                           cudaStream_t stream);

// Set the tiled kernels' shared-memory attributes on the current device
// (tet_maps.cu).
cudaError_t prepare_map_kernels();

// Free the per-relation step scratch (cg.cu).
void free_step_scratch(ebb_rel_s* rel);

// Run one implicit step (cg.cu).
ebb_status_t run_implicit_step(ebb_ctx_s* ctx, ebb_rel_s* tets, double* u, double* v,
                               const void* pinned, ebb_dtype_t pinned_dtype,
                               const ebb_step_params_t* p, ebb_cg_report_t* rep);

// Morton order, tiles and vertex index from host keys (layout.cu).  `keys`
// and `X` are the caller's order (X as 3 planes of nv); `batch` (may be null)
// gives each vertex a group id that orders tets before the Morton code
// (`known_perm`, when given, is that order already); on return
// `perm[i]` is the caller's row of internal row i, the vertex index and
// tet_perm of `tets` are on the device, and `prefix` holds the integer part
// of every tile blob (kBlobPrefix bytes per tile).
ebb_status_t build_layout(ebb_ctx_s* ctx, ebb_rel_s* tets, const std::vector<int4>& keys,
                          const std::vector<double>& X, const std::vector<int>* batch,
                          std::vector<int>& perm, std::vector<int4>& sorted_keys,
                          std::vector<unsigned char>& prefix, const std::vector<int>* known_perm = nullptr);

// Morton order of the tet centroids (grouped by the batch id of the first
// corner when `batch` is given): perm[i] = the caller's row of internal tet i.
void tet_morton_order(const std::vector<int4>& keys, const std::vector<double>& X, const std::vector<int>* batch,
                      std::vector<int>& perm);
// Tile boundaries of the internal tet order (tile t = internal tets
// [off[t], off[t+1])).
std::vector<int> tile_cut(const std::vector<int4>& sorted, int nv, int cap);
// Vertex rows for EBB_FINALIZE_RENUMBER_VERTS: with the tiles cut into
// `nchunks` consecutive ranges (as the host-buffer map cuts them), the
// vertices only one chunk touches come first, chunk by chunk, then those
// several chunks share, then unused ones, each group in order of first use
// by the Morton-ordered tets; vp[i] = the caller's vertex of row i, *n_own =
// the number of rows before the shared ones.  With `tperm_out`, also the
// tets' Morton order (tet_morton_order without batch ids), which renumbering
// the vertices leaves unchanged.
void chunked_vertex_order(const std::vector<int4>& keys, const std::vector<double>& X, int cap, int nchunks,
                          std::vector<int>& vp, int* n_own, std::vector<int>* tperm_out = nullptr);

// Pack the tile blobs (both precisions) from the host prefix and the
// device-side per-tet streams (layout.cu).
ebb_status_t build_tile_blobs(ebb_ctx_s* ctx, ebb_rel_s* tets, const std::vector<unsigned char>& prefix);
void free_layout(ebb_rel_s* tets);
// Re-cut the tiles with at most `cap` tets each and repack the blobs.
ebb_status_t rebuild_tiles(ebb_ctx_s* ctx, ebb_rel_s* tets, int cap);
// Rewrite the per-tet part of every blob in the record layout `planes`
// (the tiles stay as they are).
ebb_status_t repack_records(ebb_ctx_s* ctx, ebb_rel_s* tets, bool planes);

// Step VJP (cg.cu) and its adjoint element map (adjoint.cu).
// v_next (may be null): the step's new velocity, which replaces its forward
// solve.
ebb_status_t run_step_vjp(ebb_ctx_s* ctx, ebb_rel_s* tets, const double* u, const double* v, const double* v_next,
                          const void* pinned, ebb_dtype_t pinned_dtype, double* gu, double* gv, double* gmu,
                          double* glam, const ebb_step_params_t* p, ebb_cg_report_t* rep);
cudaError_t launch_adjoint_map(ebb_rel_s* rel, double mu0, double lam0, const double* u, const double* lv,
                               const double* w, double* acc_kl, double* acc_xq, double* gmu, double* glam, double dt,
                               cudaStream_t st);

// Batched implicit step (batched.cu).
ebb_status_t run_batched_step(ebb_ctx_s* ctx, ebb_rel_s* tets, double* u, double* v, const void* pinned,
                              const int* batch, int nmesh, const ebb_step_params_t* p, ebb_cg_report_t* reps);
void free_batch_scratch(ebb_rel_s* rel);

// Staging in the vertex-interleaved layout (reorder.cu): da/db[4 i + c] =
// a/b[c][o(i)] (b may be null); dst[k][c][o(i)] += src[k][4 i + c] for k < n
// (n <= 3); o(i) = vperm[i], or i when vperm is null.
cudaError_t interleave_fields(int nv, const int* vperm, const float* a, const float* b, float* da, float* db,
                              cudaStream_t st);
cudaError_t deinterleave_add_fields(int nv, const int* vperm, const float* const* src, float* const* dst, int n,
                                    cudaStream_t st);
// Interleaved (4-float) elements in the internal vertex order: dst[i] =
// src[vperm[i]], and dst[vperm[i]].xyz += src[i].xyz.
cudaError_t permute_vec4(int nv, const int* vperm, const float* src, float* dst, cudaStream_t st);
// Rows [r0, r1) of packed (x, y, z) FP32 triples into 4-float elements, and
// back, for the field pair (a, b); b may be null (reorder.cu).
cudaError_t xyz_to_x4(const float* sa, const float* sb, float* da, float* db, int r0, int r1, cudaStream_t st);
cudaError_t x4_to_xyz(const float* sa, const float* sb, float* da, float* db, int r0, int r1, cudaStream_t st);
cudaError_t permute_add_vec4(int nv, const int* vperm, const float* src, float* dst, cudaStream_t st);

// Vertex reordering helpers (reorder.cu).  Gather: dst[c][i] = src[c][vperm[i]];
// scatter-add: dst[c][vperm[i]] += src[c][i]; scatter: dst[c][vperm[i]] = src[c][i].
template <typename T>
cudaError_t gather_vertex_field(int nv, const int* vperm, const T* src, T* dst, cudaStream_t st);
template <typename T>
cudaError_t scatter_add_vertex_field(int nv, const int* vperm, const T* src, T* dst, cudaStream_t st);
cudaError_t scatter_vertex_field(int nv, const int* vperm, const double* src, double* dst, cudaStream_t st);
template <typename PT>
cudaError_t gather_pinned(int nv, const int* vperm, const PT* src, unsigned char* dst, cudaStream_t st);
// Morton order of vertex positions (X as 3 planes of nv): perm[i] = vertex at internal row i.
void vertex_morton_order(const std::vector<double>& X, std::vector<int>& perm);

// Edge relation, assembled stiffness and its product (edges.cu).  `keys`:
// the internal keys.  launch_assemble zeroes and assembles K(u) (u = io.u)
// in T; launch_spmv adds K w into y (3 planes, or interleaved when aos).
ebb_status_t build_edges(ebb_ctx_s* ctx, ebb_rel_s* tets, const std::vector<int4>& keys);
void free_edges(ebb_rel_s* tets);
template <typename T>
cudaError_t launch_assemble(ebb_rel_s* rel, int model, T mu0, T lam0, const MapIO<T>& io, cudaStream_t st);
template <typename T>
cudaError_t launch_spmv(ebb_rel_s* rel, const T* w, T* y, bool aos, const int* active, cudaStream_t st);

// Spring-mass system on the edge relation (springs.cu): rest lengths from
// the positions X (3 planes, FP64 or FP32), then `steps` steps in place on
// q, qd (3 planes) with per-vertex mass; *energy (host, may be null)
// receives the kinetic energy afterwards.
cudaError_t springs_init(ebb_rel_s* tets, const void* X, bool f64, cudaStream_t st);
cudaError_t springs_run(ebb_rel_s* tets, void* q, void* qd, const void* mass, bool f64, double k, double dt, int steps,
                        double* energy, cudaStream_t st);

// Build the colouring (colour.cu).
ebb_status_t build_colouring(ebb_ctx_s* ctx, ebb_rel_s* tets);
void free_colouring(ebb_rel_s* tets);

}  // namespace ebb
