/*
 * ebb.h -- C ABI of the GB300 tetrahedral-FEM map library.
 *
 * The library implements the data-parallel hot path of Ebb's relational
 * simulation model (Bernstein et al., "Ebb: A DSL for Physical Simulation on
 * CPUs and GPUs", arXiv:1506.07577) for one sm_103a GPU:
 *
 *   - relations (unordered element sets) with fields bound to them
 *     (Section 4.1, Section 5.1);
 *   - a key-field tets.v[4] linking each tetrahedron to four vertices
 *     (Section 5.1 "Key-fields", Section 5.2 "Example: FEM tetmesh");
 *   - kernels mapped over the tets relation whose per-tet results are
 *     reduced with += into vertex fields (Section 4.1, Section 6.2
 *     "Reductions");
 *   - the implicit backward-Euler step with a Jacobi-preconditioned CG solve
 *     built on those maps (Section 7.2, Vega, StVK; Section 7.3, FreeFem++,
 *     neo-Hookean).
 *
 * Conventions used by every call:
 *   - All pointers handed to the library are DEVICE pointers on the context's
 *     device unless stated otherwise.  The caller owns them; the library
 *     borrows them and never frees them (interop without marshalling,
 *     Section 4.3).
 *   - Fields are column stores (Section 6.1 "Data Layout"): a field with
 *     ncomp components over a relation of n rows occupies ncomp contiguous
 *     planes of n elements each (component c of row i at ptr[c*n + i]).
 *   - Every call returns an ebb_status_t; 0 is success.  No call aborts or
 *     throws.  ebb_last_error() gives a human-readable message for the last
 *     failure on a context.
 *   - Work is enqueued on the context's CUDA stream and is asynchronous
 *     unless stated otherwise.  Errors detected on the device (an inverted
 *     element, a bad key) are raised through a device status word that is
 *     read at the next synchronising call (ebb_ctx_sync,
 *     ebb_relation_finalize, ebb_cg_implicit_step).
 *   - Two contexts may share a device; a context must not be used from two
 *     host threads at once.
 */
#ifndef EBB_GB300_H
#define EBB_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ebb_ctx_s* ebb_ctx_t;
typedef struct ebb_rel_s* ebb_rel_t;
typedef int32_t ebb_status_t;

/* ---- status codes ------------------------------------------------------ */
#define EBB_OK                 0
#define EBB_ERR_ARG            1  /* bad argument (null, size, dtype, unknown name) */
#define EBB_ERR_KEY            2  /* key-field value < 0 or >= target size (Section 5.1) */
#define EBB_ERR_PHASE          3  /* one field used in two phases by one map (Section 4.1) */
#define EBB_ERR_INVERTED       4  /* rest tet with det(Dm) <= 0, or J <= 0 in neo-Hookean */
#define EBB_ERR_CG_BREAKDOWN   5  /* p^T A p <= 0 inside PCG */
#define EBB_ERR_NOT_CONVERGED  6  /* PCG hit max_iters above the tolerance */
#define EBB_ERR_TIMEOUT        7  /* a bounded device wait gave up */
#define EBB_ERR_CUDA           8  /* a CUDA runtime call failed */
#define EBB_ERR_STATE          9  /* call out of order (e.g. map before finalize) */
#define EBB_ERR_NOMEM         10  /* device allocation failed */

/* Field element types.  A field of ncomp components is stored as ncomp
 * contiguous planes of `size` values (plane c holds component c of every
 * row), except EBB_F32X4: FP32 3-vectors stored element by element as four
 * floats (x, y, z, and a padding value the maps ignore: reductions add zero
 * to it, EBB_MAP_ZERO_OUT zeroes it), ncomp 3, the pointer 16-byte aligned
 * -- Section 6.1's per-field
 * contiguous array of vector-valued elements, padded so that one element is
 * one 16-byte vector load or vector atomic. */
typedef enum { EBB_F32 = 1, EBB_F64 = 2, EBB_I32 = 3, EBB_U8 = 4, EBB_F32X4 = 5 } ebb_dtype_t;

/* Material models.  Section 7.2 names St. Venant-Kirchhoff, Section 7.3
 * neo-Hookean; the paper prints neither formula, the library uses the
 * textbook forms:
 *   StVK: E = (F^T F - I)/2, P = F (2 mu E + lambda tr(E) I)
 *   NH:   P = mu (F - F^-T) + lambda ln(J) F^-T                               */
typedef enum { EBB_STVK = 0, EBB_NEOHOOKEAN = 1 } ebb_model_t;

/* Element arithmetic.  EBB_PREC_F64: FP64 everywhere.  EBB_PREC_F32: element
 * maps in FP32 (Dm^-1 and volumes precomputed in FP64, stored in FP32); in
 * ebb_cg_implicit_step the CG vectors, dot products and updates stay FP64. */
typedef enum { EBB_PREC_F64 = 0, EBB_PREC_F32 = 1 } ebb_precision_t;

/* Scatter (+= reduction) strategy.
 *   ATOMIC: one thread per tet, hardware atomic adds into the vertex fields
 *           (the field reductions of Section 6.2 "Reductions").
 *   COLOR:  tets grouped by a vertex-conflict colouring, one colour at a time
 *           with plain read-modify-write; bitwise reproducible run to run
 *           (the colouring approach of Liszt discussed in Section 7.4).
 *           Needs EBB_FINALIZE_COLOR.
 *   TILED:  tets in Morton order cut into tiles; each tile gathers its
 *           distinct vertices into shared memory once, pre-reduces the
 *           per-corner results there and issues one atomic add per distinct
 *           vertex and component.
 *   GATHER: per-corner results written to a library-owned buffer (one
 *           thread per tet), then each vertex sums the entries that the
 *           inverted key-field lists for it (Section 6.1's GroupBy index,
 *           vertex -> (tet, corner) rows in increasing order), in that
 *           order, and adds the sum into its field: no atomics, bitwise
 *           reproducible run to run, no colouring needed.  The buffer
 *           (36 values per tet in the map's precision) is allocated on
 *           first use and kept with the relation.
 *   TILED_ORDERED: TILED, except that each tile stores every per-vertex
 *           sum to a partial row of its own instead of adding it atomically
 *           (a library-owned buffer of 128 rows of 12 values per tile in
 *           the map's precision, allocated on first use and kept with the
 *           tiles; a first use inside a stream capture fails with
 *           EBB_ERR_CUDA, like GATHER's); then each vertex adds
 *           its partial rows in tile order into its field.  No
 *           floating-point atomics: bitwise reproducible run to run, no
 *           colouring needed.  Not an autotuner candidate (it is the tiled
 *           pass plus a second pass).
 *   COOP:   three threads per tet (Section 8's several threads per row):
 *           thread r of a group computes row r of every per-tet matrix
 *           product and component r of every corner output, exchanging
 *           the rows it needs with its neighbours through warp shuffles;
 *           hardware atomic adds into the vertex fields.
 *   AUTO:   the autotuned choice (ebb_relation_autotune), else TILED. */
typedef enum {
  EBB_REDUCE_ATOMIC = 0,
  EBB_REDUCE_COLOR = 1,
  EBB_REDUCE_AUTO = 2,
  EBB_REDUCE_TILED = 3,
  EBB_REDUCE_GATHER = 4,
  EBB_REDUCE_TILED_ORDERED = 5,
  EBB_REDUCE_COOP = 6
} ebb_reduce_t;

/* ebb_relation_finalize flags */
#define EBB_FINALIZE_COLOR    1u  /* build the vertex-conflict colouring of tets */
#define EBB_FINALIZE_REORDER_VERTS 2u  /* number vertices internally in Morton order of
                                          their rest positions (for meshes whose vertex
                                          ids are scattered); vertex fields stay in the
                                          caller's order: maps gather inputs into the
                                          internal order and scatter outputs back, the
                                          implicit step does so once per call.  Not
                                          combinable with verts.batch; the batched step
                                          and the step VJP refuse such relations. */
#define EBB_FINALIZE_RENUMBER_VERTS 8u  /* renumber the verts relation itself in Morton
                                          order of the rest positions (Section 5.1:
                                          keys are opaque and the runtime may reorder a
                                          relation).  Every vertex field bound or read
                                          after finalize is indexed by the new row: row
                                          i holds the caller's vertex order[i] of
                                          ebb_relation_vertex_order.  verts.X (read at
                                          finalize) and tets.v keep the caller's
                                          numbering.  Maps and steps then run with no
                                          gather or scatter of vertex fields (move data
                                          into the new order once, and out when
                                          needed).  Excludes EBB_FINALIZE_REORDER_VERTS
                                          and verts.batch. */
#define EBB_FINALIZE_EDGES    4u  /* build the edge relation with self-loops and the
                                     per-tet key-field tets.e[4][4] into it (Section
                                     5.2's tetmesh domain), needed by
                                     ebb_assemble_tet_K / ebb_spmv_tet_K and
                                     EBB_STEP_ASSEMBLED */

/* map flags */
#define EBB_MAP_ZERO_OUT      1u  /* zero the output fields before reducing into them */
/* ebb_map_tet_force_Kv_host only (other calls ignore it): the host buffers
 * hold packed rows of three floats (x, y, z: 12 bytes per vertex) while the
 * bound fields are FP32 EBB_F32X4 elements.  The rows pass through a
 * library-owned device staging buffer (48 bytes per vertex, allocated on
 * first use, freed with the relation's tet data) and are widened to, or
 * narrowed from, the 4-float elements on the device, so a quarter fewer
 * bytes cross the host link. */
#define EBB_MAP_HOST_XYZ      2u
/* Testing (failure detection): the tiled map skips the bulk copy of tile 0
 * and shortens its bounded waits to about 1 ms, so the CTA that owns tile 0
 * gives up waiting, reports EBB_ERR_TIMEOUT through the device status word
 * (returned by the next synchronising call) and drains its copies; the
 * call's outputs are incomplete and the context stays usable.  Requires
 * EBB_REDUCE_TILED (or AUTO resolving to it), else EBB_ERR_ARG. */
#define EBB_MAP_TEST_DROP_TILE 0x80000000u

typedef struct {
  ebb_model_t model;
  double mu, lambda;            /* Lame parameters when the tets relation binds
                                   no per-tet "mu"/"lambda" fields */
  ebb_precision_t precision;
  ebb_reduce_t reduce;
  uint32_t flags;               /* EBB_MAP_* */
} ebb_map_opts_t;

typedef struct {
  ebb_model_t model;
  double mu, lambda;            /* as in ebb_map_opts_t */
  ebb_precision_t precision;    /* F64: all FP64.  F32: mixed (see above) */
  ebb_reduce_t reduce;
  double dt;                    /* time step */
  double gravity[3];            /* body acceleration g */
  double rho;                   /* density; lumped mass m_i = sum rho V / 4 */
  int32_t max_iters;            /* PCG iteration cap */
  double rtol;                  /* stop when ||r||_2 <= rtol ||b||_2 */
  int32_t fail_on_max_iters;    /* nonzero: hitting max_iters above rtol
                                   returns EBB_ERR_NOT_CONVERGED */
  uint32_t flags;               /* EBB_STEP_* */
} ebb_step_params_t;

/* ebb_step_params_t flags */
#define EBB_STEP_ASSEMBLED    1u  /* ebb_cg_implicit_step assembles K(x_n) once on the
                                     edge relation (EBB_FINALIZE_EDGES) and runs
                                     every CG product K p as a block-sparse product
                                     instead of the matrix-free K w map (Section
                                     7.2's Vega data layout); the other step entry
                                     points refuse it with EBB_ERR_ARG */

typedef struct {
  int32_t iters;                /* PCG iterations performed */
  double rel_residual;          /* ||r||_2 / ||b||_2 at exit (0 if b == 0) */
  ebb_status_t status;          /* same value the call returns */
} ebb_cg_report_t;

/* ---- contexts ------------------------------------------------------------ */

/* Create a context on CUDA device `device`, enqueuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Errors: EBB_ERR_ARG (null out, bad device), EBB_ERR_CUDA. */
ebb_status_t ebb_ctx_create(ebb_ctx_t* out, int device, void* cuda_stream);

/* Change the stream later calls enqueue on. */
ebb_status_t ebb_ctx_set_stream(ebb_ctx_t ctx, void* cuda_stream);

/* Destroy a context and every relation created on it, freeing the library's
 * internal device buffers (never the caller's).  NULL is accepted. */
ebb_status_t ebb_ctx_destroy(ebb_ctx_t ctx);

/* Synchronise the context's stream and return (then clear) the first error
 * raised on the device since the last synchronising call. */
ebb_status_t ebb_ctx_sync(ebb_ctx_t ctx);

/* Message describing the last failed call on ctx ("" if none).  The string is
 * owned by the context and valid until its next call. */
const char* ebb_last_error(ebb_ctx_t ctx);

/* ---- relations and fields (Section 4.1, Section 5.1) ------------------- */

/* Create a relation of `size` rows (size >= 0).  The handle lives until the
 * context is destroyed.  Errors: EBB_ERR_ARG. */
ebb_status_t ebb_relation_create(ebb_ctx_t ctx, const char* name, int64_t size,
                                 ebb_rel_t* out);

/* Bind a caller-owned device array as field `name` of relation `rel`
 * (ncomp planes of rel's size, dtype elements).  `key_target` is non-NULL
 * exactly when the field is a key-field into that relation (dtype must be
 * EBB_I32).  Rebinding a name replaces the pointer.  Fields the library
 * knows by name:
 *   verts.X       F64, 3   rest positions (read at finalize)
 *   tets.v        I32, 4   key-field into verts (tets.v[4], Section 5.2)
 *   tets.mu       F64, 1   optional per-tet Lame mu
 *   tets.lambda   F64, 1   optional per-tet Lame lambda
 * Other names are vertex fields used by maps (displacement, velocity,
 * directions, outputs).  Errors: EBB_ERR_ARG. */
ebb_status_t ebb_field_bind(ebb_rel_t rel, const char* name, ebb_dtype_t dtype,
                            int32_t ncomp, void* device_ptr, ebb_rel_t key_target);

/* Prepare a tets relation for maps: validates every key of tets.v against its
 * target (EBB_ERR_KEY, with the first bad row in the message), computes per
 * tet B = Dm^-1 and V = det(Dm)/6 in FP64 from verts.X (EBB_ERR_INVERTED if
 * det(Dm) <= 0) plus FP32 copies, snapshots per-tet Lame fields, and with
 * EBB_FINALIZE_COLOR builds the vertex-conflict colouring.  Synchronous.
 * EBB_ERR_NOMEM if device or host memory for the layout runs out (the
 * relation is then left unfinalized).  Rebinding verts.X, tets.v, tets.mu or
 * tets.lambda requires finalizing again. */
ebb_status_t ebb_relation_finalize(ebb_rel_t tets, uint32_t flags);

/* ---- maps over tets (Section 4.1 kernels, Section 6.2 reductions) ------- */
/* Vertex-field arguments are names of fields bound on the key target of
 * tets.v.  `u` is the displacement from the rest shape (x = X + u), so
 * F = Ds Dm^-1 = I + Du Dm^-1.  Field dtypes must match opts->precision
 * (F64 or F32, 3 components; in F32 either all EBB_F32 planes or all
 * EBB_F32X4 elements).  Outputs are reduce(+=) targets: the map adds
 * into them (zero them first or pass EBB_MAP_ZERO_OUT).  An output that is
 * also an input of the same map is a phase error (EBB_ERR_PHASE). */

/* f += elastic force, f = -dE/dx (per tet H = -V P(F) Dm^-T; corners 1..3 get
 * the columns of H, corner 0 minus their sum). */
ebb_status_t ebb_map_tet_forces(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                                const char* f_out, const ebb_map_opts_t* opts);

/* Kw += K(u) w, K = d^2E/dx^2 (matrix-free, per tet V dP(F; dF) Dm^-T with
 * dF = dDs(w) Dm^-1). */
ebb_status_t ebb_map_tet_Kv(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                            const char* w, const char* Kw_out,
                            const ebb_map_opts_t* opts);

/* Fused: f += force and Kw += K(u) w in one pass sharing gathers and F. */
ebb_status_t ebb_map_tet_force_Kv(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                                  const char* w, const char* f_out,
                                  const char* Kw_out, const ebb_map_opts_t* opts);

/* The fused map on host memory (Section 4.3: interop through raw memory
 * views, here on the host side).  Copies u_host and w_host into the bound
 * vertex fields u and w, runs ebb_map_tet_force_Kv(u, w, f_out, Kw_out) --
 * accumulating, or into zeroed fields with EBB_MAP_ZERO_OUT -- copies the
 * fields f_out and Kw_out into f_host and Kw_host, and returns when the
 * copies are complete.  Each host buffer holds exactly its field's bytes in
 * the field's layout (3 planes of N_v values, or N_v EBB_F32X4 elements), or,
 * with EBB_MAP_HOST_XYZ on EBB_F32X4 fields, N_v packed (x, y, z) FP32 rows;
 * page-locked host memory lets the copies run at full speed, pageable memory
 * works more slowly.  With the tiled reduction on fields the map reads in
 * place, and at least 12 tiles, the call runs in 6 consecutive tile chunks
 * (1, 3, 4, 4, 3 and 1 sixteenths of the tiles):
 * the rows chunk c reads are copied in on one library stream, its tiles are
 * mapped on the context's stream as soon as they have landed, and the rows
 * no later chunk adds to are copied out on another library stream, so the
 * copies overlap the map (fully so when consecutive tiles touch nearly
 * consecutive rows, as after EBB_FINALIZE_RENUMBER_VERTS).  The chunk plan
 * is built on the first such call after finalize or a re-tiling (a copy of
 * the internal keys to the host).  The host buffers are borrowed for the call only; the
 * device fields keep the copied and computed values afterwards.  Errors: as
 * ebb_map_tet_force_Kv (checked before anything is copied); EBB_ERR_ARG for
 * a null host buffer (with N_v > 0); EBB_ERR_PHASE if the device fields u
 * and w overlap, unless they are the same field and u_host == w_host (one
 * copy then fills it); EBB_ERR_ARG for EBB_MAP_HOST_XYZ unless the fields
 * are FP32 EBB_F32X4 elements; EBB_ERR_NOMEM if its staging buffer cannot be
 * allocated; EBB_ERR_CUDA if a copy fails. */
ebb_status_t ebb_map_tet_force_Kv_host(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                                       const char* w, const char* f_out,
                                       const char* Kw_out, const void* u_host,
                                       const void* w_host, void* f_host, void* Kw_host,
                                       const ebb_map_opts_t* opts);

/* Assembled stiffness on the edge relation (needs EBB_FINALIZE_EDGES).
 * ebb_assemble_tet_K forms K(u) in opts->precision (replacing any K
 * assembled before in that precision): one 3x3 block per edge and self-loop,
 * the sum over the tets that contain both vertices of the element blocks
 * K_ab[c][d] = V (dP(e_d b_b^T) b_a)_c -- the dP of ebb_map_tet_Kv applied to
 * one displacement component at one corner -- added with atomics (the block
 * sums are not bitwise reproducible).  The blocks are library-owned (9 values
 * per block in the assembly precision).  ebb_spmv_tet_K adds K w into Kw_out
 * with the K last assembled in opts->precision (8 lanes per vertex row,
 * fixed summation order); opts->model and ->reduce are not used by the
 * product, opts->flags may hold EBB_MAP_ZERO_OUT.  Fields as for the maps.
 * Errors: as for the maps; EBB_ERR_STATE without EBB_FINALIZE_EDGES, or for
 * a product before any assembly in that precision. */
ebb_status_t ebb_assemble_tet_K(ebb_ctx_t ctx, ebb_rel_t tets, const char* u, const ebb_map_opts_t* opts);
ebb_status_t ebb_spmv_tet_K(ebb_ctx_t ctx, ebb_rel_t tets, const char* w, const char* Kw_out,
                            const ebb_map_opts_t* opts);

/* ---- spring-mass system on the edges (Section 4.1, Figure 1) ---------- */
/* The paper's introductory example as a second workload on the same runtime;
 * the springs are the mesh's edges (needs EBB_FINALIZE_EDGES; relations
 * finalized with EBB_FINALIZE_REORDER_VERTS are refused with EBB_ERR_STATE).
 * ebb_springs_init sets every spring's rest length to the distance between
 * its ends in the vertex field `pos` (F64 or F32, 3 components), kept by the
 * library in both precisions.  ebb_springs_run advances the vertex fields q
 * (positions) and qd (velocities) by `steps` explicit steps, in place: per
 * vertex v, f_v = sum over its springs (v, h) of K (L dir - dq) with
 * dq = q_v - q_h and dir = dq / |dq| (the restoring reading of the figure,
 * whose printed dq = q_h - q_v would push a stretched spring's ends apart; a
 * zero-length dq adds nothing), then qdd = f_v / m_v, q_v += qd_v dt +
 * qdd dt^2 / 2, qd_v += qdd dt (a vertex with m <= 0 stays).  Every step
 * takes its forces from the positions at its start; each vertex sums its
 * springs in a fixed order (no atomics: bitwise reproducible).  q, qd and
 * the one-component `mass` are planes of one dtype (F64 or F32); the step's
 * arithmetic is in that dtype.  `energy` (host pointer, may be NULL)
 * receives sum m |qd|^2 / 2 after the steps (the figure's
 * measureTotalEnergy; FP64, fixed order) and makes the call synchronous.
 * Errors: EBB_ERR_ARG (fields, steps < 0, dt < 0), EBB_ERR_STATE (no edge
 * relation, no ebb_springs_init), EBB_ERR_PHASE (q, qd, mass overlap). */
ebb_status_t ebb_springs_init(ebb_ctx_t ctx, ebb_rel_t tets, const char* pos);
ebb_status_t ebb_springs_run(ebb_ctx_t ctx, ebb_rel_t tets, const char* q, const char* qd, const char* mass,
                             double k, double dt, int32_t steps, double* energy);

/* d += diag(K(u)) (closed form per tet corner and component): the Jacobi
 * preconditioner of Section 7.2. */
ebb_status_t ebb_map_tet_diagK(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                               const char* d_out, const ebb_map_opts_t* opts);

/* ---- autotuner (tile size and reduction variant) ------------------------ */
/* Section 6.2 fixes one execution mapping (one row per thread, atomic
 * reductions) and Section 8 leaves schedules and autotuning to future work;
 * this call picks the mapping of a relation by measurement.  It times the
 * K w map (the map the implicit step's CG solve runs every iteration) for
 * opts->model and opts->precision (opts->reduce and opts->flags ignored) on
 * the caller's vertex fields `u` and `w`, over the candidates: the tiled
 * variant with tiles of 128, 96 and 64 tets on the fields in place, in FP32
 * also at the best of those with the operands staged vertex-interleaved
 * (library-owned copies that let a vertex be fetched with one 16-byte copy
 * and reduced with one vector atomic, at the price of a copy in and an add
 * back per call), the atomic variant, the gather variant, the cooperative
 * variant, and the coloured variant if the relation was finalized with
 * EBB_FINALIZE_COLOR; then, at
 * the best tiled configuration, the tile blobs' per-tet data as per-field
 * planes (SoA) instead of one row record per tet (AoSoA: the fields an
 * element uses together side by side, Section 8's row-oriented storage).
 * Each candidate: 2 untimed launches, then the median of 7 launches timed
 * with CUDA events on the context's stream.  Afterwards the relation's tiles
 * use the fastest tile size (the blobs are rebuilt if it changed) and
 * EBB_REDUCE_AUTO resolves to the fastest variant for this model and
 * precision in every map and step on the relation (before any autotune it
 * resolves to EBB_REDUCE_TILED).  Results are unaffected except for the
 * order of floating-point additions.  Synchronous; allocates and frees an
 * output scratch field.  Errors: EBB_ERR_ARG / EBB_ERR_STATE as for the maps;
 * device errors of the timed maps (EBB_ERR_INVERTED) are returned. */
#define EBB_AUTOTUNE_MAX_CAND 12
typedef struct {
  int32_t reduce;       /* EBB_REDUCE_TILED, _ATOMIC, _GATHER, _COOP or _COLOR */
  int32_t tile_tets;    /* tets per tile for EBB_REDUCE_TILED, 0 otherwise */
  int32_t interleaved;  /* 1: FP32 operands staged vertex-interleaved */
  int32_t record_planes;/* 1: tile blobs hold per-tet data as field planes */
  double us;            /* median duration of one K w map call, microseconds */
} ebb_autotune_cand_t;

typedef struct {
  int32_t reduce;       /* variant EBB_REDUCE_AUTO now selects */
  int32_t tile_tets;    /* tets per tile of the relation's layout now */
  int32_t interleaved;  /* FP32 tiled maps now stage operands vertex-interleaved */
  int32_t record_planes;/* tile blobs now hold per-tet data as field planes */
  int32_t ncand;
  ebb_autotune_cand_t cand[EBB_AUTOTUNE_MAX_CAND];
} ebb_autotune_report_t;

ebb_status_t ebb_relation_autotune(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                                   const char* w, const ebb_map_opts_t* opts,
                                   ebb_autotune_report_t* report);

/* Set by hand what ebb_relation_autotune would choose: EBB_REDUCE_AUTO
 * resolves to `reduce` (TILED, TILED_ORDERED, ATOMIC, GATHER, COOP or COLOR) for `model` and
 * `precision`;
 * the tiles are re-cut to at most `tile_tets` tets (1..128) if that differs;
 * `flags` holds EBB_TUNE_INTERLEAVED (the FP32 vertex-interleaved staging of
 * the tiled maps) and EBB_TUNE_RECORD_PLANES (tile blobs with per-tet data as
 * field planes; without it, row records).  Synchronous.  Errors: EBB_ERR_ARG
 * (out-of-range value), EBB_ERR_STATE (not finalized, or COLOR without
 * EBB_FINALIZE_COLOR). */
#define EBB_TUNE_INTERLEAVED    1u
#define EBB_TUNE_RECORD_PLANES  2u
ebb_status_t ebb_relation_set_tuning(ebb_ctx_t ctx, ebb_rel_t tets, int32_t model,
                                     int32_t precision, int32_t reduce, int32_t tile_tets,
                                     int32_t flags);

/* Layout of a finalized tets relation as the maps see it (read only, host
 * side): how many tiles the tiled variants walk and how many tets each holds
 * at most, how many colours the coloured variant launches, whether FP32 tiled
 * maps stage their operands vertex-interleaved, whether vertices are
 * renumbered internally, and the variant EBB_REDUCE_AUTO resolves to per
 * [model][precision] (-1: not tuned, AUTO means TILED).  Errors:
 * EBB_ERR_ARG (null argument), EBB_ERR_STATE (not finalized). */
typedef struct {
  int64_t n_tets, n_verts;
  int32_t ntiles;          /* tiles of the tiled variants */
  int32_t tile_tets;       /* tets per tile at most */
  int32_t ncolours;        /* colours (0 without EBB_FINALIZE_COLOR) */
  int32_t interleaved;     /* FP32 tiled maps stage operands vertex-interleaved */
  int32_t reordered;       /* 1: EBB_FINALIZE_REORDER_VERTS, 2: EBB_FINALIZE_RENUMBER_VERTS */
  int32_t record_planes;   /* tile blobs hold per-tet data as field planes */
  int32_t tuned[2][2];     /* autotuned reduce per [model][precision], -1 none */
} ebb_relation_info_t;

ebb_status_t ebb_relation_info(ebb_ctx_t ctx, ebb_rel_t tets, ebb_relation_info_t* info);

/* Row order of the verts relation after finalize: order[i] = the caller's
 * vertex (its row before finalize, the numbering of verts.X and tets.v) now
 * held in row i of every vertex field.  Identity unless the relation was
 * finalized with EBB_FINALIZE_RENUMBER_VERTS (EBB_FINALIZE_REORDER_VERTS
 * keeps fields in the caller's order).  `order` is a HOST array of n =
 * N_v entries.  Synchronous.  Errors: EBB_ERR_ARG (n != N_v, null order),
 * EBB_ERR_STATE (not finalized). */
ebb_status_t ebb_relation_vertex_order(ebb_ctx_t ctx, ebb_rel_t tets, int32_t* order, int64_t n);

/* ---- implicit step (Section 7.2, Section 7.3) --------------------------- */

/* One linearised backward-Euler step, in place on the F64 vertex fields
 * `u` (displacement) and `v` (velocity):
 *   A = M + dt^2 K(x_n),  b = dt (f(x_n) + M g - dt K(x_n) v_n),
 *   A dv = b by Jacobi PCG from dv = 0 (rows/cols of pinned vertices
 *   removed), v += dv, u += dt v.
 * `pinned` names a U8 or I32 one-component vertex field (nonzero = pinned),
 * or is NULL.  The PCG loop runs on the device without host round trips
 * except one status read per batch of iterations.  Synchronous; fills
 * *report (may be NULL).  Errors: EBB_ERR_CG_BREAKDOWN,
 * EBB_ERR_NOT_CONVERGED (if requested), EBB_ERR_INVERTED, plus argument
 * errors.  After a solve that ran, u and v are advanced with the last CG
 * iterate even when the call returns one of these three errors. */
ebb_status_t ebb_cg_implicit_step(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                                  const char* v, const char* pinned,
                                  const ebb_step_params_t* params,
                                  ebb_cg_report_t* report);

/* Vector-Jacobian product of one implicit step (the adjoint; St.
 * Venant-Kirchhoff, FP64 only).  `u`, `v` name the state at the START of the
 * step (read only; the step is re-solved internally from it).  `gu`, `gv`
 * name F64 vertex fields holding dL/du', dL/dv' of a scalar loss L with
 * respect to the step's outputs; on return they hold dL/du, dL/dv.
 * `gmu`, `glam` name F64 one-component fields bound on the tets relation (in
 * the caller's tet order) into which dL/dmu and dL/dlambda of each tet are
 * ADDED; either may be NULL.  With x = X + u, A = M + dt^2 K(x) and v' the
 * step's new velocity:
 *   A lam = dL/dv' + dt dL/du'  (pinned rows zero; same PCG, same operator)
 *   dL/du = dL/du' - dt K lam - dt^2 d/dx[lam^T K(x) v']
 *   dL/dv = dL/dv' + dt dL/du' - dt^2 K lam
 *   dL/dtheta += dt d/dtheta[lam^T f] - dt^2 d/dtheta[lam^T K v']  per tet.
 * The report describes the adjoint solve.  Synchronous.  Errors as for
 * ebb_cg_implicit_step, plus EBB_ERR_ARG for another model or precision and
 * EBB_ERR_PHASE if u, v, gu, gv overlap. */
ebb_status_t ebb_cg_implicit_step_vjp(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                                      const char* v, const char* pinned, const char* gu,
                                      const char* gv, const char* gmu, const char* glam,
                                      const ebb_step_params_t* params,
                                      ebb_cg_report_t* report);

/* The same vector-Jacobian product for a caller that already holds the
 * step's new velocity: `v_next` names an F64 vertex field with v' (for
 * example from the forward replay of a checkpointed rollout).  The forward
 * solve is skipped (dv = v' - v); the adjoint solve, the adjoint element map
 * and the outputs are as in ebb_cg_implicit_step_vjp, which this equals to
 * the forward solve's tolerance when v_next is that step's result.  Errors as
 * ebb_cg_implicit_step_vjp; EBB_ERR_ARG for a null v_next, EBB_ERR_PHASE if
 * v_next overlaps u, v, gu or gv. */
ebb_status_t ebb_cg_implicit_step_vjp_at(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                                         const char* v, const char* v_next, const char* pinned,
                                         const char* gu, const char* gv, const char* gmu,
                                         const char* glam, const ebb_step_params_t* params,
                                         ebb_cg_report_t* report);

/* Batched form: one implicit step for each of many independent meshes
 * stored in one verts/tets relation pair (for example hundreds of small
 * meshes of uneven sizes; the per-mesh step is exactly the one above).
 * `batch` names an I32 one-component vertex field giving each vertex its mesh
 * id in [0, nbatch); ids must be non-decreasing along verts (each mesh's
 * vertices contiguous) and every id must occur.  Bind the field as
 * "batch" before ebb_relation_finalize so tets are ordered mesh by mesh and
 * a tet joining two meshes is rejected (EBB_ERR_KEY).  Every element map
 * runs as one launch over all meshes; CG scalars, convergence and iteration
 * counts are per mesh (a converged mesh stops updating while others go on).
 * `pinned` must be a U8 field or NULL.  reports (may be NULL) receives nbatch
 * entries.  Synchronous.  Returns the first failing mesh's status (its
 * message names the mesh), else EBB_OK. */
ebb_status_t ebb_cg_implicit_step_batched(ebb_ctx_t ctx, ebb_rel_t tets, const char* u,
                                          const char* v, const char* pinned,
                                          const char* batch, int32_t nbatch,
                                          const ebb_step_params_t* params,
                                          ebb_cg_report_t* reports);

/* ---- implicit step without device allocation ---------------------------- */
/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory -- code running where cudaMalloc is not
 * allowed or not wanted (a host framework that owns every device byte and
 * hands out fixed arenas, real-time loops that must not hit the allocator, or
 * contexts created before any allocator is set up).  Contexts, relations and
 * finalize all allocate, so this call takes plain device arrays instead:
 *   keys    I32, 4 planes of n_tets (tets.v[4]; each key in [0, n_verts))
 *   X       F64, 3 planes of n_verts: rest positions
 *   u, v    F64, 3 planes of n_verts: displacement and velocity, updated in
 *           place exactly as ebb_cg_implicit_step updates them
 *   pinned  U8, n_verts (nonzero = pinned), or NULL
 * on the current CUDA device, enqueued on `cuda_stream` (NULL = legacy
 * default stream); the call is synchronous.  Only params->precision ==
 * EBB_PREC_F64 and uniform material (params->mu, params->lambda) are
 * supported, and the scatter is always the atomic one.
 * Its working memory is one fixed array in the library's device image
 * (about 2.8 MB, held on every device that loads the library until the
 * process exits), so sizes are capped: n_verts <=
 * EBB_NOALLOC_MAX_VERTS and n_tets <= EBB_NOALLOC_MAX_TETS, else EBB_ERR_ARG
 * before any work is enqueued.  The call neither allocates nor frees device
 * memory.  Every call looks up the array's device address on the current
 * device; the first call on a device also loads the library's device code
 * there, so make it before any stream capture.  Every call reuses the same
 * array, so two calls whose work overlaps on the GPU (other streams, other
 * host threads) race and corrupt each other; the call clears what must start
 * at zero.
 * Errors: EBB_ERR_ARG, EBB_ERR_KEY, EBB_ERR_INVERTED, EBB_ERR_CG_BREAKDOWN,
 * EBB_ERR_NOT_CONVERGED (if requested), EBB_ERR_CUDA.  There is no context,
 * so no message: only the status code.  A bad key or an inverted rest tet is
 * found before anything is written, and u, v are then left untouched; after
 * a solve that ran (EBB_ERR_INVERTED from an element of the deformed state,
 * EBB_ERR_CG_BREAKDOWN, EBB_ERR_NOT_CONVERGED) u and v have been advanced with
 * the last CG iterate, as ebb_cg_implicit_step does. */
#define EBB_NOALLOC_MAX_VERTS 4096
#define EBB_NOALLOC_MAX_TETS 24576
ebb_status_t ebb_cg_implicit_step_noalloc(void* cuda_stream, int32_t n_verts, int32_t n_tets,
                                          const int32_t* keys, const double* X, double* u,
                                          double* v, const uint8_t* pinned,
                                          const ebb_step_params_t* params,
                                          ebb_cg_report_t* report);

#ifdef __cplusplus
}
#endif
#endif /* EBB_GB300_H */
