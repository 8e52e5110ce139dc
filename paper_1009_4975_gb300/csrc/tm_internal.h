// Internal declarations shared by the translation units of libtm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdlib>
#include <deque>
#include <exception>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tm.h"
#include "element.cuh"

namespace amr {

// Operator kernel geometry: one CTA per block of consecutive (Morton-ordered)
// elements.  A block's "local nodes" are the non-hanging nodes its elements
// touch directly or through a hanging corner's masters.
#ifndef TM_BLOCK_ELEMS
#define TM_BLOCK_ELEMS 256
#endif
constexpr int kBlockElems = TM_BLOCK_ELEMS;   // elements per block (ragged last block)
constexpr int kMaxLocal = 1024;      // local nodes per block
constexpr int kSlotRow = 25;         // per-element row of the operator's result buffer (24 + 1 pad)
constexpr int kFoldBit = 0x8000;     // inverse-list entry names a hanging node to fold in
constexpr int kQuarterBit = 0x4000;  // ... whose weight is 1/4 (else 1/2)

// ---------------------------------------------------------------- host tables
struct HostMesh {
  int nx = 0, ny = 0, nz = 0, L = 0;
  double h0 = 0;
  uint32_t dirichlet_faces = 0;
  double E0 = 1, Emin = 0, nu = 0.3, penal = 3;
  int64_t Ne = 0, Nn = 0;
  std::vector<int32_t> leaf;          // 4 per element, canonical order
  std::vector<int64_t> perm;          // canonical element -> input leaf
  std::vector<uint64_t> node_key;     // Morton key per node (sorted)
  std::vector<int32_t> node_xyz;      // 3 per node
  std::vector<int32_t> conn;          // 8 per element
  std::vector<uint8_t> nflag;         // bit 0 Dirichlet, bit 1 hanging
  std::vector<int32_t> hang_node;     // ascending
  std::vector<int32_t> hang_master;   // 4 per hanging node, -1 padded, ascending
  std::vector<int32_t> hang_index;    // node -> hanging index or -1
  int64_t n_dirichlet = 0, n_free_nodes = 0;

  // operator blocks (runs of consecutive canonical elements outside the bricks).  Local node ids of a
  // block: regular nodes first (shared ones, then interior), then the hanging
  // nodes its elements use.  The inverse list of a local node names the
  // (element, corner) slots it fills -- entry e_local * kSlotRow + 3 k, the slot's
  // offset in the per-element result buffer (< 0x4000) -- and, for a regular node,
  // the hanging nodes it is a master of -- entry kFoldBit | (kQuarterBit if the
  // hanging node has 4 masters) | hanging index.
  int32_t nblk = 0, max_local = 0;
  std::vector<int32_t> gen_elem;      // the elements outside the bricks, ascending
  std::vector<int32_t> blk_elem;      // 2 per block: its range [u0, u1) of gen_elem
  std::vector<int32_t> blk_node;      // nblk+1: regular local node ranges in lnode
  std::vector<int32_t> blk_shared;    // nblk: regular local nodes [0, shared) are shared
  std::vector<int32_t> blk_slot;      // nblk+1: the block's shared nodes' range in lslot
  std::vector<int32_t> blk_hang;      // nblk+1: hanging ranges in hent
  std::vector<int32_t> blk_iptr;      // nblk+1: ranges in iptr (local nodes + 1)
  std::vector<int32_t> blk_inv;       // nblk: base of the block's entries in inv
  std::vector<int32_t> lnode;         // regular local node -> global node
  std::vector<int32_t> lslot;         // shared local node -> its partial's position (node-major CSR)
  std::vector<uint16_t> hent;         // 4 per hanging local node: masters' local ids (0xFFFF pad)
  std::vector<uint16_t> iptr;         // inverse-list offsets, relative to blk_inv[b]
  std::vector<uint16_t> inv;          // inverse-list entries
  std::vector<uint16_t> lcorner;      // 8 per element: local ids of its corners within its block
  std::vector<uint8_t> brec;          // per-block records (see mesh_host.cpp, 16-byte aligned)
  std::vector<int32_t> rec_off;       // nblk+1: record ranges in 16-byte units
  std::vector<int32_t> rec_skip;      // nblk: 16-byte units of lcorner and elist (not staged)
  int32_t max_rec_bytes = 0;
  int32_t max_rec_stage = 0;          // largest staged part: header + the sections from lnode on
  // bricks (mesh_host.cpp, section 6a): aligned 4x4x4 runs of 64 equal-level elements taken by
  // the brick pass; their 5x5x5 node lattice is node (a, b, c) at a + 5 b + 25 c
  int32_t nbrick = 0;
  std::vector<int32_t> brick_e0;      // first element of each brick
  std::vector<int32_t> brick_node;    // 125 per brick: global node, bit 31 = Dirichlet
  std::vector<uint8_t> brick_hax;     // 125 per brick: 0 regular, else the axes (bits 0-2) a hanging
                                      // node interpolates along (masters one lattice step away)
  std::vector<int32_t> brick_out;     // 125 per brick: -1 the brick owns the node, >= 0 its partial's
                                      // position (node-major CSR), -2 hanging (folded into masters)
  std::vector<uint32_t> brick_fold;   // 125 per brick: lattice neighbours folded into a regular node
  std::vector<int32_t> brick_tab;     // 384 per brick: the device copy (brick.cuh)
  int64_t nslot = 0;                  // partials of block- and brick-shared nodes
  // second pass over shared nodes
  std::vector<int32_t> sh_node;       // shared node ids
  std::vector<int32_t> sh_ptr;        // CSR: partials of shared node i are [sh_ptr[i], sh_ptr[i+1])
  std::vector<int32_t> sh_of_node;    // node -> shared-node index or -1
  // Jacobi diagonal: node-centric CSR of (element, coefficient-triple index)
  std::vector<int32_t> dg_ptr;        // Nn+1
  std::vector<int32_t> dg_elem;
  std::vector<uint16_t> dg_q;
  std::vector<double> dg_tab;         // 3 per distinct triple
  // the reference element matrix (unit cube, E = 1), host copy
  std::vector<double> K0;             // 24 x 24
  std::vector<double> modal;          // 8 x 3 x 3 blocks of K0 in the butterfly basis (element.cuh)
  std::vector<int32_t> cellmap;       // finest cell (x fastest) -> canonical element
};

// Returns "" on success or an error message.
std::string build_host_mesh(const tm_mesh_desc &d, HostMesh &m);
std::string adapt_leaves(const HostMesh &m, const int8_t *mark, const double *rho, std::vector<int32_t> &leaves,
                         std::vector<double> &rho_out);
void reference_stiffness(double nu, double *K0 /* 576 */);
uint64_t morton3(uint32_t x, uint32_t y, uint32_t z);

// ---------------------------------------------------------------- device state
template <typename T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
};

struct DeviceMesh {
  int64_t Ne = 0, Nn = 0, nh = 0, nsh = 0;
  int32_t nblk = 0;
  int fx = 0, fy = 0, fz = 0;         // finest grid extents
  int L = 0;
  double h0 = 0, hmin = 0;
  double E0 = 1, Emin = 0, penal = 3, nu = 0.3;
  double modal[72] = {};              // element matrix blocks (element.cuh)
  double k0diag = 0;
  double volume = 0;                  // |Omega|
  int64_t n_free = 0;
  int32_t *leaf = nullptr;            // 4 per element (canonical)
  int32_t *cellmap = nullptr;         // finest cell -> element (canonical)
  int32_t *conn = nullptr;            // 8 per element (canonical)
  uint8_t *nflag = nullptr;
  int32_t *hang_node = nullptr;
  int32_t *hang_master = nullptr;     // 4 per
  int32_t *blk_elem = nullptr, *blk_node = nullptr, *blk_shared = nullptr, *blk_slot = nullptr,
          *blk_hang = nullptr, *blk_iptr = nullptr, *blk_inv = nullptr;
  int32_t *lnode = nullptr, *lslot = nullptr;
  uint16_t *hent = nullptr, *iptr = nullptr, *inv = nullptr;
  int32_t max_local = 0;
  uint4 *brec = nullptr;
  int32_t *rec_off = nullptr;
  int32_t *rec_skip = nullptr;
  int32_t max_rec_bytes = 0, max_rec_stage = 0;
  int32_t resident_cta32 = 0, resident_cta64 = 0;  // block-pass CTAs resident on the GPU (record prefetch distance)
  int32_t nbrick = 0;                 // bricks (HostMesh): CTAs nblk .. of the block pass take 4 each
  int32_t *brick_tab = nullptr;       // 384 per brick (brick.cuh)
  int32_t *sh_node = nullptr, *sh_ptr = nullptr;
  int32_t *sh_of_node = nullptr;      // node -> shared-node index, -1 when one block owns it
  int32_t *dg_ptr = nullptr, *dg_elem = nullptr;
  uint16_t *dg_q = nullptr;
  double *dg_tab = nullptr;
  int64_t nslot = 0;
  std::vector<void *> owned;
  int64_t bytes = 0;
};

// CTAs of the operator's block pass: the blocks, then the bricks four to a CTA
inline int apply_ctas(const DeviceMesh &m) { return m.nblk + (m.nbrick + 3) / 4; }

// Two-level preconditioner (kernels_coarse.cu): levels of the uniform vertex lattice, level 0
// the base grid.  Lattice vectors hold 3 values per node, x fastest, clamped nodes at 0.
constexpr int kMaxCoarseLevels = 12;
struct SolveScalars;
constexpr int kMaxCoarsestDofs = 1200;   // the coarsest level is solved by a dense inverse (host Cholesky)
struct CoarseLevel {
  int X = 0, Y = 0, Z = 0, nodes = 0;    // cells per axis, (X+1)(Y+1)(Z+1) nodes
  double H = 0;                          // cell side
  double *mom = nullptr;                 // cells x 27 moments of E (FP64)
  float *K = nullptr;                    // cells x 24 x 24 cell matrices
  float *dinv = nullptr;                 // 3 * nodes: inverse l1 row sums (0 at clamped nodes)
  float *b = nullptr, *x = nullptr, *x2 = nullptr, *t = nullptr;   // kMaxRhs cases x 3 * nodes each
};
struct CoarseHierarchy {
  int nlev = 0;
  unsigned faces = 0;                    // the mesh's clamped faces
  CoarseLevel lev[kMaxCoarseLevels];
  int32_t *cell_elem = nullptr;          // 2 per base cell: its leaves' canonical range
  int32_t *cptr = nullptr, *cnode = nullptr;   // per base cell: the mesh nodes it owns (CSR)
  int32_t nseg = 0;                      // restriction segments: runs of <= 64 of a cell's nodes
  int32_t *seg_ptr = nullptr;            // nseg + 1: segment s covers cnode[seg_ptr[s], seg_ptr[s+1])
  int32_t *seg_cell = nullptr;           // nseg: its cell
  int32_t *cseg = nullptr;               // base cells + 1: cell c's segments [cseg[c], cseg[c+1])
  int32_t *ncell = nullptr;              // per mesh node: its base cell
  uint32_t *code = nullptr;              // per mesh node: position in the cell, bit 31 = no unknowns
  uint32_t *ccode = nullptr;             // the same codes in cnode order (read beside cnode)
  // the moment -> cell-matrix coefficients (27 x 576, coarse_moment_matrices), as the upper
  // triangle by entry: qent[u] = i | j << 5 | nonzeros << 10, then per entry the
  // moments with a nonzero coefficient (qidx, ascending) and the coefficients (qval)
  int32_t *qent = nullptr;
  uint8_t *qidx = nullptr;
  double *qval = nullptr;
  float *part = nullptr;                 // kMaxRhs cases x segments x 24: partial restrictions
  double *Kc64 = nullptr;                // coarsest level's cell matrices in FP64
  float *Ainv = nullptr;                 // coarsest level: dense inverse over all its DOFs
  std::vector<double> Kc_host;           // host copy of Kc64 (inverse formed on the host)
  std::vector<float> Ainv_host;          // the inverse, kept until its upload has completed
  std::vector<void *> owned;
  int64_t bytes = 0;
};
// Host side (coarse_host.cpp): level shapes (empty string) or why the mesh has no usable
// hierarchy; the per-node and per-cell tables; the moment matrices; the coarsest inverse.
std::string coarse_shapes(const HostMesh &m, std::vector<int> &shapes);
void coarse_tables(const HostMesh &m, std::vector<int32_t> &cell_elem, std::vector<int32_t> &cptr,
                   std::vector<int32_t> &cnode, std::vector<int32_t> &ncell, std::vector<uint32_t> &code);
constexpr int kSegNodes = 64;
constexpr int kCellUpper = 300;   // entries of the upper triangle of a 24 x 24 cell matrix
constexpr int kCellNnz = 27;      // room per entry for its nonzero moment coefficients
void coarse_segments(const std::vector<int32_t> &cptr, std::vector<int32_t> &seg_ptr, std::vector<int32_t> &seg_cell,
                     std::vector<int32_t> &cseg);
void coarse_moment_matrices(double nu, std::vector<double> &Q);
std::string coarse_dense_inverse(const std::vector<double> &Kc, int X, int Y, int Z, unsigned faces,
                                 std::vector<float> &Ainv);
cudaError_t coarse_setup_launch(const DeviceMesh &m, CoarseHierarchy &h, const double *rho, cudaStream_t s);
// Load cases c0 .. c0 + nv - 1 per launch (sc: all cases' CG scalars, may be NULL outside a solve);
// fine vectors of consecutive cases are r_ld (ld) floats apart.
cudaError_t coarse_restrict_launch(const DeviceMesh &m, const CoarseHierarchy &h, const float *r, int64_t r_ld,
                                   bool first_sweep, const struct SolveScalars *sc, int c0, int nv, cudaStream_t s);
cudaError_t coarse_vcycle_launch(const CoarseHierarchy &h, int nu, const struct SolveScalars *sc, int c0, int nv,
                                 cudaStream_t s, int *launches);
cudaError_t coarse_finish_launch(const CoarseHierarchy &h, int mode, struct SolveScalars *sc, int c0, int nv,
                                 double *partials, int pstride, unsigned int *tickets, cudaStream_t s);
cudaError_t coarse_pupdate_launch(const DeviceMesh &m, const CoarseHierarchy &h, float *p, const float *r,
                                  int64_t ld, const float *dinv, int mode, const struct SolveScalars *sc, int c0,
                                  int nv, cudaStream_t s);
cudaError_t coarse_prolong_launch(const DeviceMesh &m, const CoarseHierarchy &h, const float *v, float *y,
                                  cudaStream_t s);
cudaError_t coarse_level_apply_launch(const CoarseHierarchy &h, int l, const float *x, float *y, cudaStream_t s);
cudaError_t coarse_first_sweep_launch(const CoarseHierarchy &h, cudaStream_t s);

// Learned initial guess (kernels_learn.cu): the voxel grid of level g and its gather tables.
struct LearnTables {
  int g = -1, X = 0, Y = 0, Z = 0, hv = 0;   // grid level, cells, cell side in finest units
  int32_t *nxyz = nullptr;               // 3 per mesh node (finest units)
  int32_t *vptr = nullptr, *vnode = nullptr;   // nodes grouped by their lower stencil cell (CSR)
  double *pf = nullptr;                  // 3 x cells scratch of the restrictions
  std::vector<void *> owned;
  int64_t bytes = 0;
};
cudaError_t learn_input_launch(const DeviceMesh &m, const LearnTables &t, const double *rho, const double *f,
                               double *pf, double *partials, unsigned int *ticket, double *s_dev, float *x,
                               cudaStream_t st);
cudaError_t learn_guess_launch(const DeviceMesh &m, const LearnTables &t, const float *out, double s, double *u0,
                               cudaStream_t st);
cudaError_t learn_grad_launch(const DeviceMesh &m, const LearnTables &t, const double *au0, const double *f, double s,
                              double *pf, float *dout, cudaStream_t st);
cudaError_t adam_launch(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st);

// Work buffers of one context (sized for the current mesh).
struct Work {
  double *part64 = nullptr;    // 3 * nslot, partial sums of shared nodes (FP64 operator)
  float *part32 = nullptr;     // 3 * nslot (FP32 operator)
  double *ce64 = nullptr;      // Ne, coefficients E_e h_e (canonical order)
  float *ce32 = nullptr;
  double *red = nullptr;       // reduction partials
  double *scal = nullptr;      // device scalars
  unsigned int *ticket = nullptr;  // last-block counters
  int *status = nullptr;       // device status word
  int8_t *mark_tmp = nullptr;  // Ne, intermediate adaptation marks
  double4_32a *octab = nullptr;    // Ne, the OC update's per-element table (on first use)
  float *part_multi = nullptr; // kMaxRhs * 3 * nslot, partials of the multi-vector operator (on first use)
  // multi-load CG (on first use): per load case x, r, p, q (FP32) and the FP64 residual,
  // CG scalars, element-energy partials
  float *mvec = nullptr;       // 4 kinds (x, r, p, q) x kMaxRhs load cases x 3 Nn (kind-major)
  double *mr64 = nullptr;      // kMaxRhs * 3 Nn
  struct SolveScalars *msc = nullptr;   // kMaxRhs
  double *mdotp = nullptr;     // kMaxRhs * nblk
  double *mred = nullptr;      // kMaxRhs x 16 SMs: per-case reduction partials
  unsigned int *mticket = nullptr;   // 4 x kMaxRhs: per-case last-CTA tickets
  // solver vectors (3 * Nn)
  double *r = nullptr, *p = nullptr, *q = nullptr, *dinv = nullptr, *d = nullptr;
  float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *dinv32 = nullptr, *x32 = nullptr;
  int64_t nred = 0;
  std::vector<void *> owned;
  int64_t bytes = 0;
};

}  // namespace amr

struct tm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  bool has_mesh = false;
  amr::HostMesh host;
  amr::DeviceMesh dm;
  amr::Work w;
  amr::CoarseHierarchy coarse;   // two-level preconditioner (allocated on first use per mesh)
  amr::LearnTables learn;        // learned initial guess (allocated on first use per mesh and grid)
  bool coarse_ready = false;     // its operators match the last density set up
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // profiling (tm_profile): kernel launch count and CUDA-event operator timing
  bool prof_on = false;
  int64_t launches = 0;
  tm_profile_data prof = tm_profile_data();
  struct Pending {
    cudaEvent_t e0, e1;
    int kind;          // 1: FP32 operator, 0: FP64 operator
    bool graph_owned;  // recorded by a captured graph (kept with it)
  };
  std::vector<Pending> ev_pending;
  std::vector<cudaEvent_t> ev_free;
  // CG batches captured as CUDA graphs, replayed on the context's own stream
  struct Graph {
    const void *key[4] = {};
    int count = 0;
    int precond = 0, nu = 0;   // two-level batches differ from Jacobi batches
    int launches = 0;          // kernels per replay
    bool prof = false;
    cudaGraphExec_t exec = nullptr;
    std::vector<Pending> ev;
  };
  std::deque<Graph> graphs;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_coarse = nullptr;   // the coarsest level's cell matrices reached the host
  bool capturing = false;
};

// Host threads the library may use at once: the hardware's, at most 16, and at most the positive
// integer in the environment variable TM_HOST_THREADS when it holds one (read at every call).
inline int host_thread_limit() {
  int hw = (int)std::thread::hardware_concurrency();
  if (hw <= 0) hw = 1;
  if (const char *env = std::getenv("TM_HOST_THREADS")) {
    char *end = nullptr;
    const long v = std::strtol(env, &end, 10);
    if (end != env && *end == 0 && v > 0) hw = (int)std::min<long>(v, hw);
  }
  return std::min(hw, 16);
}

// The handler of the C-ABI entry points' function-try-blocks (call it only inside a catch): a C++
// exception must not cross the C boundary, so it becomes a status -- TM_ENOMEM for a failed host
// allocation (std::bad_alloc, std::length_error), TM_EINVAL for anything else -- and the context,
// when there is one, keeps its message.
inline int exception_status(tm_ctx *ctx) noexcept {
  int code = TM_EINVAL;
  const char *what = "unexpected C++ exception";
  try {
    throw;
  } catch (const std::bad_alloc &) {
    code = TM_ENOMEM;
    what = "host memory allocation failed";
  } catch (const std::length_error &) {
    code = TM_ENOMEM;
    what = "host array size out of range";
  } catch (const std::exception &e) {
    what = e.what();
  } catch (...) {
  }
  if (ctx) {
    try {
      ctx->err = what;
    } catch (...) {
    }
  }
  return code;
}

namespace amr {
// device-side launchers of the operator file; each returns the launch's cudaError_t
cudaError_t launch_coeff(const DeviceMesh &m, const Work &w, const double *rho, cudaStream_t s);
struct SolveScalars;
// y = C^T K C x.  With dot_partials: also x^T A x (element energies); with sc:
// alpha = sc->rz / (x^T A x) computed by the last CTA of the block pass (ticket:
// its counter).
template <typename T>
cudaError_t launch_apply(const DeviceMesh &m, const T *ce, const T *x, T *y, T *part, double *dot_partials,
                         SolveScalars *sc, unsigned int *ticket, bool zero_hanging, const int *done,
                         cudaStream_t s);
cudaError_t launch_diag(const DeviceMesh &m, const double *ce, double *d, double *dinv, float *dinv32,
                        cudaStream_t s);
cudaError_t launch_expand(const DeviceMesh &m, const double *u, double *uf, cudaStream_t s);
int shared_grid(int64_t n);
// The block pass alone: y is complete at nodes owned by one block; shared nodes'
// contributions are left in `part` (CSR order, see DeviceMesh::sh_ptr).
template <typename T>
cudaError_t launch_apply_blocks(const DeviceMesh &m, const T *ce, const T *x, T *y, T *part, double *energy_partials,
                                SolveScalars *sc, unsigned int *ticket, const int *done, cudaStream_t s);

// Static scratch of the no-allocation operator entry point (kernels_apply.cu).
constexpr int64_t kStaticElems = int64_t(1) << 21;   // coefficients: meshes up to 2,097,152 elements
constexpr int64_t kStaticSlots = int64_t(1) << 21;   // shared-node partials: up to 2,097,152
constexpr int kStaticMaxDevices = 64;
cudaError_t static_scratch(int device, float **ce, float **part);
// Multiprocessors of the current device (queried once per device); grid-stride kernels cap
// their grids at a multiple of it.
int device_sms();
cudaError_t launch_coeff_f32(const DeviceMesh &m, const double *rho, float *ce32, cudaStream_t s);
cudaError_t apply_residency(const DeviceMesh &m, int *resident32, int *resident64);
// U-Net layers (kernels_unet.cu)
cudaError_t unet_conv_fwd(const float *x, const float *w, const float *b, float *y, int N, int Ci, int Co, int X,
                          int Y, int Z, int K, bool relu, cudaStream_t s);
cudaError_t unet_relu_bwd(const float *y, float *g, int64_t n, cudaStream_t s);
cudaError_t unet_conv_bwd(const float *x, const float *w, const float *dy, float *dx, bool dx_accumulate, float *dw,
                          float *db, int N, int Ci, int Co, int X, int Y, int Z, int K, cudaStream_t s);
cudaError_t unet_pool_fwd(const float *x, float *y, int64_t NC, int X, int Y, int Z, cudaStream_t s);
cudaError_t unet_spread(const float *in, float *out, int64_t NC, int X, int Y, int Z, bool pool_adjoint,
                        bool accumulate, cudaStream_t s);
cudaError_t unet_gather8(const float *in, float *out, int64_t NC, int X, int Y, int Z, cudaStream_t s);
cudaError_t unet_channels_copy(const float *src, int Cs, int sc0, float *dst, int Cd, int dc0, int nc, int N,
                               int64_t S, bool accumulate, cudaStream_t s);
// several vectors at once (kernels_multi.cu)
constexpr int kMaxRhs = 8;
size_t apply_multi_smem_bytes(const DeviceMesh &m, int nr);
struct SolveScalars;
cudaError_t launch_apply_multi(const DeviceMesh &m, int nr, const float *ce, const float *x, float *y, float *part,
                               double *dotp, SolveScalars *sc, unsigned int *ticket, cudaStream_t s);
// adaptation (kernels_amr.cu)
cudaError_t launch_amr_mark(const DeviceMesh &m, const double *rho, double rho_solid, double r_amr, int8_t *tmp,
                            int8_t *mark, cudaStream_t s);
cudaError_t launch_transfer(const DeviceMesh &m, const double *u_full, const int32_t *pts, int64_t n, double *out,
                            int *bad, cudaStream_t s);
cudaError_t launch_design_difference(const DeviceMesh &m, const double *rho1, const int32_t *leaves2, int64_t n2,
                                     const double *rho2, int32_t *map2, double *partials, unsigned int *ticket,
                                     double *out, cudaStream_t s);
}  // namespace amr
