/*
 * tm.h -- C ABI of the GB300 hot path for SIMP topology optimisation on a
 * dynamically refined, 2:1-balanced octree hex mesh (Wang, de Sturler,
 * Paulino, "Dynamic adaptive mesh refinement for topology optimization").
 *
 * The library solves the paper's state equation K(rho) u = f (Sec. 3, Eq. 1)
 * on B8 (trilinear hex) elements with element-constant density and SIMP
 * stiffness E_e = Emin + rho_e^p (E0 - Emin) (Eq. 2, Emin = 0 is the paper's
 * form), eliminates hanging-node DOFs by the interpolation of Sec. 6 (Eq. 6-9),
 * and provides the remaining steps of one optimisation iteration: compliance
 * sensitivities, the volume-weighted filter of Eq. 5 and the optimality-
 * criteria update.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Status: every function returns TM_OK (0) or a TM_E* code; the message of
 *   the last failure is available from tm_last_error().  Nothing falls back to
 *   the host: a missing or failing GPU is an error.  No C++ exception leaves the
 *   library: a failed host allocation inside a call returns TM_ENOMEM, and a host
 *   thread that cannot be started leaves its share of the work to the calling one.
 * - Memory: pointers named *_dev are caller-owned device memory on the
 *   context's device; all other pointers are caller-owned host memory that is
 *   only read (or written, for outputs) during the call.  The library copies
 *   what it keeps.
 * - Streams: work is enqueued on the stream given to tm_create / tm_set_stream
 *   (a cudaStream_t, NULL = legacy default).  Device outputs are valid once that
 *   stream reaches them.  Calls that return a host scalar synchronise the
 *   stream before returning.
 * - Node vectors ("A-space"): length 3*Nn doubles, node-major, component
 *   fastest (x, y, z), nodes in canonical order.  Entries at hanging and
 *   Dirichlet DOFs are ignored on input and written as 0 on output; the
 *   remaining n_free entries are the unknowns of the reduced system
 *   A = C^T K C (Eq. 7 with the constrained DOFs eliminated; the paper's Eq. 8
 *   keeps them with a unit diagonal and yields the same u).
 * - Full vectors: length 3*Nn with hanging DOFs interpolated (Eq. 9) and
 *   Dirichlet DOFs at their prescribed value 0.
 * - Element vectors: length Ne doubles in canonical element order.
 * - Canonical orders: elements by the Morton key of their anchor, nodes by
 *   the Morton key of their coordinates (bit i of x, y, z at bits 3i, 3i+1,
 *   3i+2); local corner k = i + 2j + 4m of an element sits at anchor + s(i,j,m).
 */
#ifndef TM_H
#define TM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TM_OK 0
#define TM_EINVAL 1          /* bad argument or invalid mesh                      */
#define TM_ECUDA 2           /* CUDA runtime error (message has the CUDA string)  */
#define TM_ENOTCONVERGED 3   /* solver hit max_iter before rtol                   */
#define TM_ENONFINITE 4      /* NaN/Inf met in a reduction                        */
#define TM_ETIMEOUT 5        /* a bounded device-side wait gave up                */
#define TM_ENOMEM 6          /* device or host allocation failed                  */
#define TM_ESTATE 7          /* call out of order (e.g. no mesh uploaded)         */

#define TM_PREC_FP64 0       /* every step in FP64                                */
#define TM_PREC_MIXED 1      /* FP32 CG with FP64 reliable updates                */
#define TM_PREC_FP32 1

typedef struct tm_ctx tm_ctx;

/* A mesh: the box [0, nx h0] x [0, ny h0] x [0, nz h0] split into base cells of
 * side h0, refined up to max_level.  Leaves are given on the finest integer grid
 * (unit h0 / 2^max_level): leaf (ix, iy, iz, l) is the cube of side
 * 2^(max_level - l) units anchored at (ix, iy, iz). */
typedef struct {
  int32_t nx, ny, nz;
  int32_t max_level;
  double h0;
  int64_t n_leaves;
  const int32_t *leaves;      /* host, 4 * n_leaves: ix, iy, iz, level          */
  uint32_t dirichlet_faces;   /* bit 2*axis + side: that face is clamped (u = 0) */
  double E0, Emin, nu, penal; /* SIMP material, Eq. 2                            */
} tm_mesh_desc;

typedef struct {
  int64_t Ne, Nn;             /* elements, nodes                                  */
  int64_t n_hanging;          /* hanging nodes                                    */
  int64_t n_dirichlet;        /* Dirichlet nodes (hanging ones included)          */
  int64_t n_free;             /* unknowns: 3 * (nodes neither hanging nor clamped) */
  int32_t n_blocks;           /* element blocks of the operator kernel            */
  int32_t max_local;          /* largest local-node count of a block              */
  int64_t n_shared;           /* nodes touched by more than one block or brick    */
  int64_t device_bytes;       /* device memory held for this mesh                 */
  int32_t max_block_bytes;    /* table bytes of the largest block (shared memory) */
  int32_t n_bricks;           /* 4x4x4 equal-level bricks taken by the brick pass  */
} tm_mesh_info;

typedef struct {
  double rtol;                /* stop when ||f - A u||_2 <= rtol ||f||_2          */
  int32_t max_iter;           /* CG iterations in all                             */
  int32_t precision;          /* TM_PREC_FP64 or TM_PREC_MIXED                    */
  double inner_rtol;          /* mixed: FP32 residual reduction between two FP64
                                 residual replacements (<= 0: 0.1)                */
  int32_t check_every;        /* iterations between host convergence checks       */
  int32_t no_graphs;          /* 0: each batch of check_every CG iterations is a   */
                              /* CUDA graph replayed on a library stream; 1: plain */
                              /* launches on the context's stream                   */
  int32_t precond;            /* TM_PRECOND_JACOBI (0) or TM_PRECOND_TWOLEVEL (1) */
  int32_t smooth_sweeps;      /* two-level: l1-Jacobi sweeps before and after the  */
                              /* coarse-grid step on each level (<= 0: 1)         */
} tm_solve_opts;

/* Preconditioners of tm_pcg_solve.  TM_PRECOND_JACOBI: the diagonal of A (the rescaling of
 * Sec. 5).  TM_PRECOND_TWOLEVEL (TM_PREC_MIXED only): the diagonal plus a Galerkin coarse
 * correction on the vertex lattice of the base grid, applied through a V-cycle (see
 * tm_coarse_setup).  The paper keeps the slowly converging part of the spectrum from solve
 * to solve in a recycled Krylov subspace (Sec. 5); the coarse space takes that role here. */
#define TM_PRECOND_JACOBI 0
#define TM_PRECOND_TWOLEVEL 1

typedef struct {
  int32_t iterations;         /* CG iterations performed                          */
  int32_t sweeps;             /* mixed: FP64 residual replacements; FP64: 1        */
  double rel_residual;        /* final ||f - A u|| / ||f|| evaluated in FP64      */
  double seconds;             /* device time of the solve (CUDA events)           */
  int32_t fp64_applies;       /* FP64 operator applications                       */
  int32_t fp32_applies;       /* FP32 operator applications                       */
  int32_t coarse_levels;      /* two-level: lattice levels of the V-cycle; else 0 */
  int32_t pad_;
  double setup_seconds;       /* two-level: host time of the per-density set-up   */
} tm_solve_stats;

/* Counters of tm_profile / tm_profile_read. */
typedef struct {
  int64_t launches;           /* kernels this context launched since tm_profile    */
  int64_t apply32_count;      /* FP32 operator applications timed                  */
  int64_t apply64_count;      /* FP64 operator applications timed                  */
  double apply32_ms;          /* their summed CUDA-event time (both passes)        */
  double apply64_ms;
} tm_profile_data;

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream`
 * (cudaStream_t or NULL).  *out receives the context; TM_ECUDA if the device is
 * unusable. */
int tm_create(tm_ctx **out, int device, void *cuda_stream);
int tm_destroy(tm_ctx *ctx);
int tm_set_stream(tm_ctx *ctx, void *cuda_stream);
const char *tm_last_error(tm_ctx *ctx);

/* Build the mesh tables of Sec. 6 from a leaf set and upload them (paper
 * Sec. 4 marks/refines, Sec. 6 Fig. 3 limits incompatibility to one level).
 * Rejects with TM_EINVAL: leaves out of range or misaligned, overlapping or
 * non-covering leaf sets, sets that are not 2:1 balanced (any two leaves
 * whose closures meet differ by at most one level), 2^29 leaves or more, and
 * meshes whose tables would need a 32-bit offset above 2^31 - 1 (3 Nn, the
 * Jacobi-diagonal entries, the shared-node partials or the block records).
 * Replaces any previous mesh.  `info` (may be NULL) receives the sizes. */
int tm_mesh_upload(tm_ctx *ctx, const tm_mesh_desc *d, tm_mesh_info *info);

/* Copy the integer tables to host arrays (any may be NULL):
 * perm[Ne]        canonical element i is input leaf perm[i];
 * node_xyz[3*Nn]  node coordinates on the finest grid;
 * conn[8*Ne]      node id of corner k of element e at conn[8e + k];
 * hang_node[nh]   hanging node ids, ascending;
 * hang_master[4*nh] their masters ascending (-1 padded; 2 = edge, 4 = face);
 * node_flags[Nn]  bit 0 Dirichlet, bit 1 hanging. */
int tm_mesh_tables(tm_ctx *ctx, int64_t *perm, int32_t *node_xyz, int32_t *conn,
                   int32_t *hang_node, int32_t *hang_master, uint8_t *node_flags);

/* Host-only construction of the same integer tables (no device, no context):
 * the tables tm_mesh_upload builds, for inspection and testing on machines
 * without a GPU.  On failure returns TM_EINVAL and writes a message into err
 * (err_len bytes, may be 0).  info->device_bytes is 0.
 * Host threads: tm_mesh_upload, tm_tables_build, the adaptation's new leaf set
 * (tm_amr_adapt, tm_tables_adapt) and the two-level preconditioner's host part
 * (its per-mesh tables and the coarsest level's dense inverse, in the first solve
 * on a mesh and in tm_coarse_setup) run on up to 16 host threads, one per 65,536
 * items at most; the environment variable TM_HOST_THREADS (a positive integer,
 * read at every call) lowers the limit.  Every table and error is the same for
 * any number of threads. */
typedef struct tm_tables tm_tables;
int tm_tables_build(const tm_mesh_desc *d, tm_tables **out, tm_mesh_info *info, char *err, int err_len);
/* Same layout as tm_mesh_tables. */
int tm_tables_copy(const tm_tables *t, int64_t *perm, int32_t *node_xyz, int32_t *conn, int32_t *hang_node,
                   int32_t *hang_master, uint8_t *node_flags);
void tm_tables_free(tm_tables *t);
/* Host-only export of the operator's block tables, for checking them without a GPU:
 * rec_off[n_blocks + 1] (record ranges in 16-byte units), brec[*rec_bytes] (the
 * per-block records the operator kernel stages: a header of 16 int32 -- first
 * element, elements, regular and shared local nodes, hanging local nodes, inverse
 * entries, byte offsets of the lslot, hent, iptr, inv, lcorner, lnode and elist sections,
 * three zeros -- then those sections; elist names the block's elements, ascending, which
 * are the elements outside the bricks (tm_tables_bricks) taken in order), modal[72] (the element matrix of the unit cube in the
 * symmetry-adapted basis: 8 blocks of 3 x 3, row-major, block s couples the modes
 * s^1, s^2, s^4 of components 0, 1, 2), sh_node[n_shared] and sh_ptr[n_shared + 1]
 * (block-shared nodes and the ranges of their partials).  Any pointer may be NULL;
 * call with brec NULL to learn *rec_bytes first. */
int tm_tables_operator(const tm_tables *t, int32_t *rec_off, uint8_t *brec, double *modal, int32_t *sh_node,
                       int32_t *sh_ptr, int64_t *rec_bytes);
/* Host-only export of the brick tables (info->n_bricks bricks; any pointer may be NULL).  A brick
 * is an aligned cube of 4x4x4 elements of one level, 64 consecutive elements in the canonical
 * (Morton) order, element e0[i] + morton(x, y, z) at cube position (x, y, z); the blocks hold the
 * other elements.  Its 5x5x5 node lattice, node (a, b, c) at a + 5 b + 25 c: node[125 i + ...]
 * (global node id, bit 31 set at Dirichlet nodes), hax[...] (0 for a regular node; for a hanging
 * node the axes, bits 0-2, along which it interpolates its masters, the lattice nodes one step
 * away), out[...] (-1: the node's result is written to y by this brick alone; >= 0: the position
 * of its partial in the shared-node pass, as sh_ptr ranges; -2: hanging), fold[...] (for a regular
 * node, the lattice neighbours that are hanging nodes it is a master of: bit 2 a + (step > 0) the
 * neighbour one step along axis a, hanging along a; bit 6 + 4 p + 2 (step1 > 0) + (step0 > 0) the
 * diagonal neighbour in coordinate plane p = (x, y), (x, z), (y, z), hanging in that plane). */
int tm_tables_bricks(const tm_tables *t, int32_t *e0, int32_t *node, uint8_t *hax, int32_t *out, uint32_t *fold);
/* Host-only export of the Jacobi-diagonal tables of tm_jacobi_diag (Sec. 5), node-major:
 * the diagonal of C^T K(rho) C at a free node n, component c, is the sum over
 * j in [ptr[n], ptr[n + 1]) of c_e tab[3 q[j] + c] with e = elem[j] (ascending within a node)
 * and c_e = (Emin + rho_e^penal (E0 - Emin)) h_e, h_e the element's edge length; tab holds the
 * distinct triples v^T K0_cc v of the unit cube's matrix K0 (E = 1), v the node's weights on
 * the element's corners (1 at its own corner; 1/2 or 1/4 at the corners it is a master of),
 * tab[0..2] the triple of a corner that is its own node.  Sizes: ptr[Nn + 1],
 * elem[*n_entries], q[*n_entries], tab[3 *n_triples].  Any pointer may be NULL; call with
 * them NULL to learn the sizes first. */
int tm_tables_diag(const tm_tables *t, int32_t *ptr, int32_t *elem, uint16_t *q, double *tab, int64_t *n_entries,
                   int64_t *n_triples);

/* Host-only evaluation of a finite-element field of the tables' mesh at integer points
 * (the warm start after remeshing: the old displacement at the new mesh's nodes, see
 * Sec. 5 on mapping the solution onto the updated mesh).  u_full (host, 3 * Nn doubles,
 * hanging entries interpolated as tm_expand writes them) is trilinear on every leaf and
 * continuous; out (host, 3 * n_points) receives its value at points (host, 3 * n_points
 * int32 finest-grid coordinates, inside the closed box; TM_EINVAL otherwise). */
int tm_tables_transfer(const tm_tables *t, const double *u_full, int64_t n_points, const int32_t *points,
                       double *out);

/* Device form of tm_tables_transfer on the context's (old) mesh: the field u_full_dev (device,
 * 3 Nn doubles of the uploaded mesh, hanging entries interpolated, as tm_expand gives it)
 * evaluated at points_dev (device, 3 * n_points int32 finest-grid coordinates, e.g. the nodes
 * of the adapted mesh) into out_dev (device, 3 * n_points doubles): the warm start of the solve
 * after remeshing (Sec. 5 solves a sequence of systems; the paper maps data to the updated mesh,
 * Sec. 4).  Synchronises the stream; TM_EINVAL if a point lies outside the closed box. */
int tm_transfer_displacement(tm_ctx *ctx, const double *u_full_dev, int64_t n_points, const int32_t *points_dev,
                             double *out_dev);

/* Host-only form of tm_amr_adapt on built tables (marks and rho on the host, in
 * the tables' element order); same rules, outputs and errors. */
int tm_tables_adapt(const tm_tables *t, const int8_t *mark, const double *rho, int64_t capacity,
                    int32_t *leaves_out, double *rho_out, int64_t *n_out);


/* f_dev (A-space) = C^T f_full where f_full holds the given nodal point loads
 * (Eq. 7 right-hand side).  node_xyz: host, 3 per load, must be mesh nodes
 * (TM_EINVAL otherwise); comp in {0,1,2}; loads on hanging nodes are folded
 * into their masters. */
int tm_build_rhs(tm_ctx *ctx, int64_t n_loads, const int32_t *node_xyz, const int32_t *comp,
                 const double *val, double *f_dev);

/* y = C^T K(rho) C x on the A-space (Eq. 6-7), FP64 arithmetic. */
int tm_apply_K(tm_ctx *ctx, const double *rho_dev, const double *x_dev, double *y_dev);

/* Same operator in FP32 arithmetic on FP32 A-space vectors (the inner operator
 * of TM_PREC_MIXED). */
int tm_apply_K_f32(tm_ctx *ctx, const double *rho_dev, const float *x_dev, float *y_dev);

/* The FP32 operator on nrhs vectors at once (1 <= nrhs <= 8; several load cases of one
 * design): y_dev[r] = C^T K(rho) C x_dev[r] (Eq. 6-9), x_dev and y_dev each nrhs
 * consecutive A-space vectors of 3 * Nn floats (device).  Each y_dev[r] is the result
 * of tm_apply_K_f32 on x_dev[r] bit for bit; the operator tables are staged once per
 * block for all vectors.  Its partial-sum scratch (4 * 3 floats per block-shared node
 * partial) is allocated on the first call for the uploaded mesh. */
int tm_apply_K_f32_multi(tm_ctx *ctx, int nrhs, const double *rho_dev, const float *x_dev, float *y_dev);

/* The FP32 operator of tm_apply_K_f32 for callers that cannot allocate device
 * memory when they call: services whose device memory is a fixed pool reserved
 * at start-up, host applications whose allocator forbids cudaMalloc/cudaFree
 * after initialisation, and plug-ins that may only use buffers the host hands
 * them.  It has no counterpart in the paper.
 * It allocates nothing: its scratch (the element coefficients and the
 * shared-node partials) lives in one statically sized device array of 32 MiB
 * that every GPU loading the library holds until the process exits.  The caller
 * passes rho, x and y as for tm_apply_K_f32; the uploaded mesh must have at most
 * 2,097,152 elements and 2,097,152 shared-node partials, else TM_EINVAL names
 * the sizes.  The first call on a device looks up the array's device address
 * (module set-up, once per device under a lock, with that device current).  All
 * calls share the one array and every call
 * overwrites all of it that it reads, so nothing carries over between calls;
 * calls that overlap on the GPU (other streams, other contexts of the same
 * device) race on it, so the caller serialises them.  tm_profile does not time
 * this entry point (it counts its launches only). */
int tm_apply_K_f32_static(tm_ctx *ctx, const double *rho_dev, const float *x_dev, float *y_dev);

/* d_dev = diag(C^T K(rho) C) on the A-space (1 at constrained DOFs): the
 * diagonal D of the rescaling D^-1/2 K D^-1/2 of Sec. 5. */
int tm_jacobi_diag(tm_ctx *ctx, const double *rho_dev, double *d_dev);

/* Solve C^T K(rho) C u = f by Jacobi-preconditioned CG (equivalent to CG on the
 * diagonally rescaled system of Sec. 5), warm-started from u_dev (Sec. 5).
 * TM_PREC_FP64: every step in FP64.  TM_PREC_MIXED: CG with the FP32 operator and
 * FP32 vectors (dot products accumulated in FP64) and reliable updates: whenever the
 * FP32 residual has dropped by inner_rtol, the FP32 correction is added to u in FP64
 * and the residual is replaced by the FP64 true residual f - A u, keeping the search
 * direction (made orthogonal to the new residual); convergence is always judged on the
 * FP64 true residual.  Returns TM_ENOTCONVERGED (u holds the last iterate) when
 * max_iter is reached, TM_ENONFINITE on NaN/Inf. `stats` may be NULL; stats->sweeps
 * counts the FP64 residual replacements. */
int tm_pcg_solve(tm_ctx *ctx, const double *rho_dev, const double *f_dev, double *u_dev,
                 const tm_solve_opts *opts, tm_solve_stats *stats);

/* Several independent solves at once (one design and load case per context, each
 * context with its own mesh): solve i is tm_pcg_solve(ctxs[i], rho_dev[i], f_dev[i],
 * u_dev[i], opts, &stats[i]) and gives the same result bit for bit; the solves run
 * concurrently, one host thread per context, so that small meshes (which leave most
 * of the GPU idle alone) share it.  The contexts must be distinct (TM_EINVAL
 * otherwise); for the solves to overlap on the GPU each context needs its own
 * non-default stream.  stats (n entries) and status (n entries, each solve's
 * return code) may be NULL.  Returns TM_OK when every solve did, else the first
 * non-OK code; each context's tm_last_error describes its own failure. */
int tm_pcg_solve_batch(int n, tm_ctx *const *ctxs, const double *const *rho_dev, const double *const *f_dev,
                       double *const *u_dev, const tm_solve_opts *opts, tm_solve_stats *stats, int *status);

/* Several load cases of one design at once (1 <= nrhs <= 8; TM_PREC_MIXED only):
 * f_dev and u_dev hold nrhs consecutive A-space vectors (device), u_dev the warm starts
 * on entry.  The load cases iterate in lockstep; each has its own CG scalars and
 * reliable updates, and gets the same u and iteration count as tm_pcg_solve with the
 * same options, bit for bit.  Per iteration one operator pass serves all cases
 * (tm_apply_K_f32_multi), one launch updates all cases and, with TM_PRECOND_TWOLEVEL, one
 * launch sequence applies the coarse correction of all cases (the level matrices are read
 * once for all); cases that reached their stopping point skip the work.  Unless
 * opts->no_graphs, each batch of check_every lockstep iterations is a CUDA graph replayed on
 * a library stream.  stats: nrhs entries (may be NULL); their seconds field is the time of the
 * whole call.  Work buffers for 8 load cases are allocated on the first call for the
 * uploaded mesh. */
int tm_pcg_solve_multi(tm_ctx *ctx, int nrhs, const double *rho_dev, const double *f_dev, double *u_dev,
                       const tm_solve_opts *opts, tm_solve_stats *stats);

/* ---- Two-level preconditioner (TM_PRECOND_TWOLEVEL).  An extension with no paper
 * counterpart: it takes the role of the recycled Krylov subspace of Sec. 5, removing the
 * smooth, slowly converging part of the error by a projection onto a coarse space.
 *   M^-1 r = D^-1 r + P0 V_0(P0^T r)
 * Levels: level 0 is the vertex lattice of the base grid (nx x ny x nz cells of side h0);
 * level l+1 halves every cell count of level l and exists while all three are even and
 * level l has more than 64 cells; the last level is solved directly and must have at most
 * 1200 unknowns (TM_EINVAL otherwise).  A lattice vector of a level with X x Y x Z cells
 * holds 3 floats per node, node i + (X+1)(j + (Y+1)k), component fastest; entries at nodes
 * on clamped faces are 0.  P0 is the trilinear interpolation of level-0 values at the free
 * mesh nodes (the coarse space is nested in the finite-element space because every leaf
 * lies in one base cell, consistent with the hanging-node interpolation of Eq. 6); level
 * operators are Galerkin, A_0 = P0^T A P0 and A_(l+1) = P^T A_l P with nodal
 * interpolation P; V_0 is a V-cycle with `nu` l1-Jacobi sweeps before and after the
 * coarse-grid step on each level.  All device vectors below are FP32, caller-owned, and
 * stream-ordered on the context's stream. */

/* Build the level operators for the density rho_dev (Ne doubles, canonical order): cell
 * matrices from the moments of E(x) over each cell, l1-Jacobi diagonals and the coarsest
 * dense inverse (on the host; synchronises the stream).  levels_out (host, may be NULL):
 * the number of levels; shapes_out (host, 3 per level, may be NULL): their cell counts.
 * tm_pcg_solve with TM_PRECOND_TWOLEVEL does this itself.  TM_EINVAL when the base grid
 * does not coarsen to a small enough level. */
int tm_coarse_setup(tm_ctx *ctx, const double *rho_dev, int32_t *levels_out, int32_t *shapes_out);

/* Copy level `level`'s cell matrices (X*Y*Z cells x 24 x 24 floats, cells x fastest, local
 * DOF 3 q + c of corner q = a + 2b + 4c) into K_dev.  TM_ESTATE before tm_coarse_setup. */
int tm_coarse_cells(tm_ctx *ctx, int level, float *K_dev);

/* y_dev = A_level x_dev on lattice vectors of that level (TM_ESTATE before set-up). */
int tm_coarse_apply(tm_ctx *ctx, int level, const float *x_dev, float *y_dev);

/* b0_dev = P0^T r_dev: r_dev an FP32 A-space vector (3 Nn), b0_dev a level-0 lattice vector. */
int tm_coarse_restrict(tm_ctx *ctx, const float *r_dev, float *b0_dev);

/* y_dev = P0 v0_dev: the FP32 A-space vector of the level-0 lattice vector v0_dev (0 at
 * hanging and clamped DOFs). */
int tm_coarse_prolong(tm_ctx *ctx, const float *v0_dev, float *y_dev);

/* x0_dev = V_0(b0_dev) with nu >= 1 sweeps (level-0 lattice vectors). */
int tm_coarse_vcycle(tm_ctx *ctx, const float *b0_dev, float *x0_dev, int nu);

/* u_full = C u (Eq. 9): hanging DOFs interpolated, Dirichlet DOFs 0. */
int tm_expand(tm_ctx *ctx, const double *u_dev, double *u_full_dev);

/* dc_e = -p rho_e^(p-1) (E0 - Emin) h_e u_e^T K0 u_e (compliance sensitivity of
 * Sec. 3) from a full vector; *compliance_out (host, may be NULL) receives
 * sum_e E_e h_e u_e^T K0 u_e, which equals f^T u (Eq. 1) at convergence. */
int tm_sensitivity(tm_ctx *ctx, const double *rho_dev, const double *u_full_dev, double *dc_dev,
                   double *compliance_out);

/* Element filters over centre distances below rmin with H_de = rmin - dist
 * (Eq. 4), self included:
 * mode 0: Eq. 5, out_e = sum_d rho_d H_de V_d x_d / (rho_e sum_d H_de V_d);
 * mode 1: density filter, out_e = sum_d H_de V_d x_d / sum_d H_de V_d.
 * rmin is limited to 4 finest cells (TM_EINVAL beyond). */
int tm_filter(tm_ctx *ctx, const double *rho_dev, const double *x_dev, double rmin, int mode,
              double *out_dev);

/* Optimality-criteria update (Sec. 3): rho_new = clamp(rho (max(-dc,0)/(lambda V_e))^eta,
 * max(rho_min, rho - move), min(1, rho + move)) with lambda such that
 * sum rho_new V_e = volfrac * |Omega|: found on the device by a safeguarded Newton search on
 * the volume (a piecewise linear function of lambda^-eta), each step bracketing the root,
 * until the relative lambda bracket is below 1e-12 (lambda is the bracket's midpoint) or a
 * step hits the target volume exactly.
 * *change_out (host, may be NULL) receives max |rho_new - rho|. */
int tm_oc_update(tm_ctx *ctx, const double *rho_dev, const double *dc_dev, double volfrac, double move,
                 double eta, double rho_min, double *rho_new_dev, double *change_out);

/* Dynamic adaptation, step 1 (Sec. 4): mark_dev (device, Ne int8, element order
 * of tm_mesh_tables) receives +1 (refine), 0 (keep) or -1 (derefine).
 * An element is solid when rho_e >= rho_solid; it is marked +1 when it is solid
 * or the centre of a solid element lies at a distance below r_amr from its
 * centre, else -1; +1 at the finest level and -1 at level 0 become 0.  Then the
 * two sweeps of Sec. 4: a -1 survives only when all 8 siblings are leaves
 * marked -1, and only when every leaf touching the parent box ends, after its
 * own refinement, at most one level finer than the parent (coarsenings of
 * neighbours are not counted).  r_amr is limited to 4 finest cells (TM_EINVAL
 * beyond), like the filter radius.  rho_dev: device, Ne doubles. */
int tm_amr_mark(tm_ctx *ctx, const double *rho_dev, double rho_solid, double r_amr, int8_t *mark_dev);

/* Dynamic adaptation, step 2 (Sec. 4, with the balancing of Sec. 6): the leaves
 * of the adapted mesh from marks (device, Ne int8) and densities (device, Ne
 * doubles).  Elements marked +1 split into 8 children that inherit rho; a
 * family of 8 siblings all marked -1 merges into its parent, whose rho is the
 * mean of the 8 (summed in sibling order, x fastest); then leaves are refined
 * (children inherit rho) until touching leaves differ by at most one level.
 * Output on the host, in Morton order: leaves_out[4*capacity] as (ix, iy, iz,
 * level) like tm_mesh_desc, rho_out[capacity]; *n_out receives the leaf count
 * even when it exceeds capacity (then TM_EINVAL and nothing is written).  Runs
 * on the host after copying the marks and densities back (synchronises the
 * stream).  TM_EINVAL for +1 at the finest level, -1 at level 0, or a -1 family
 * that is not 8 sibling leaves all marked -1. */
int tm_amr_adapt(tm_ctx *ctx, const int8_t *mark_dev, const double *rho_dev, int64_t capacity,
                 int32_t *leaves_out, double *rho_out, int64_t *n_out);

/* Design difference of Eq. 10 between the uploaded mesh with rho_dev (device,
 * Ne doubles) and another design on the same box and maximum level
 * (leaves_other: host, 4*n_other int32 as in tm_mesh_desc, any order;
 * rho_other: host, n_other doubles): *d_out (host) = sum_c |rho1_c - rho2_c| /
 * sum_c rho1_c over the cells c of the finest grid, each cell taking the
 * density of the leaf covering it (all cells have the same volume).  Allocates
 * device memory for the other design and a cell map (4 bytes per finest cell)
 * for the duration of the call and synchronises the stream.  TM_EINVAL when the
 * other leaves do not tile the box exactly once. */
int tm_design_difference(tm_ctx *ctx, const double *rho_dev, int64_t n_other, const int32_t *leaves_other,
                         const double *rho_other, double *d_out);

/* ---- Learned initial guess (no counterpart in the paper): a 3D U-Net ------------
 * Per level i < levels: two 3x3x3 convolutions (zero padding, bias) each followed by
 * ReLU, channels[i] features; 2x2x2 average pooling between levels; on the way up,
 * nearest 2x upsampling, concatenation [upsampled, skip] along channels and the two
 * convolutions of that level; a 1x1x1 output convolution to c_out channels.
 * Activations: n x C x x x y x z FP32, contiguous (device); x, y, z multiples of
 * 2^(levels - 1).  Parameters: one FP32 array (device), tm_unet_param_count floats,
 * per convolution its weights (Cout x Cin x k x k x k) then its bias, in the order
 * encoder levels 0..levels-1, decoder levels levels-2..0, output.  Workspace:
 * tm_unet_workspace_floats floats (device), caller-owned.
 * tm_unet_forward: y = net(x); keeps the activations in the workspace.
 * tm_unet_backward: given dy = dL/dy, writes dL/dparams (and dL/dx when dx is not
 * NULL); needs the workspace of a tm_unet_forward with the same params and x.
 * Direct CUDA-core kernels with fixed summation orders.  TM_EINVAL for a bad
 * description or null pointers.  The count functions return -1 for a bad one. */
typedef struct {
  int32_t levels;             /* 1..6                                               */
  int32_t channels[6];        /* features per level                                 */
  int32_t c_in, c_out;
  int32_t n, x, y, z;         /* batch and grid                                     */
} tm_unet_desc;
int64_t tm_unet_param_count(const tm_unet_desc *d);
int64_t tm_unet_workspace_floats(const tm_unet_desc *d);
int tm_unet_forward(tm_ctx *ctx, const tm_unet_desc *d, const float *params, const float *x, float *y, float *ws);
int tm_unet_backward(tm_ctx *ctx, const tm_unet_desc *d, const float *params, const float *x, const float *dy,
                     float *dparams, float *dx, float *ws);

/* ---- Transfers and optimiser of the learned initial guess (no paper counterpart).  The
 * voxel grid of level g (0 <= g <= max_level) has X = nx 2^g, Y = ny 2^g, Z = nz 2^g cells
 * of side h0 / 2^g (at least 2 per axis); voxel arrays are channel-major with z fastest
 * (c, i, j, k), FP32, device.  P is the trilinear interpolation of cell-centred values at the
 * mesh nodes, with the lower cell index clamped to [0, n - 2] per axis (linear extrapolation in
 * the boundary half-cells); P^T is its adjoint on the A-space.  Tables are built on the first
 * call for a mesh and grid level (host work). */

/* Network input x_dev (4 channels): channel 0 the volume average of rho over each voxel,
 * channels 1-3 P^T f_dev (f_dev: the A-space load vector, as tm_build_rhs gives it) divided by
 * s = max |P^T f|, returned in *s_out (host; synchronises the stream).  TM_EINVAL when s = 0. */
int tm_learn_input(tm_ctx *ctx, const double *rho_dev, const double *f_dev, int g, float *x_dev, double *s_out);

/* u0_dev (A-space FP64, 0 at constrained DOFs) = s P(out_dev): the initial guess from the
 * network output out_dev (3 channels). */
int tm_learn_guess(tm_ctx *ctx, const float *out_dev, double s, int g, double *u0_dev);

/* dout_dev (3 channels) = s P^T (au0_dev - f_dev): the gradient of the energy loss
 * 0.5 u0^T A u0 - f^T u0 with respect to the network output when au0_dev = A u0 (tm_apply_K). */
int tm_learn_output_grad(tm_ctx *ctx, const double *au0_dev, const double *f_dev, double s, int g, float *dout_dev);

/* One Adam step (Kingma and Ba, 2015) on n FP32 parameters with their gradients, first and
 * second moment estimates m_dev and v_dev (zero before step 1), step >= 1 counting from 1. */
int tm_adam_step(tm_ctx *ctx, int64_t n, float *params_dev, const float *grads_dev, float *m_dev, float *v_dev,
                 int step, float lr, float beta1, float beta2, float eps);

/* Instrumentation (no counterpart in the paper): tm_profile(ctx, 1) resets the
 * counters and starts timing every operator application with a CUDA-event
 * pair on the context's stream (both passes of the operator; applications a CG
 * batch enqueued past convergence return at once and are not counted);
 * tm_profile(ctx, 0) stops timing.  tm_profile_read synchronises the stream
 * and returns the counters. */
int tm_profile(tm_ctx *ctx, int enable);
int tm_profile_read(tm_ctx *ctx, tm_profile_data *out);

#ifdef __cplusplus
}
#endif
#endif /* TM_H */
