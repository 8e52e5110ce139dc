// C ABI of libtm (declared in include/tm.h): argument checks, device memory of
// the mesh tables and work buffers, and the host-side drivers of the solvers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <chrono>
#include <thread>
#include <type_traits>
#include <vector>

#include "pcg.cuh"
#include "tm_internal.h"
#include "topopt.cuh"

using namespace amr;

namespace {

int fail(tm_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

#define TM_CUDA(ctx, ...)                                                                   \
  do {                                                                                      \
    cudaError_t _e = (__VA_ARGS__);                                                         \
    if (_e != cudaSuccess)                                                                  \
      return fail(ctx, TM_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(_e)); \
  } while (0)

#define TM_CHECK_CTX(ctx)                                                                   \
  do {                                                                                      \
    if (!(ctx)) return TM_EINVAL;                                                           \
    cudaError_t _e = cudaSetDevice((ctx)->device);                                          \
    if (_e != cudaSuccess) return fail(ctx, TM_ECUDA, cudaGetErrorString(_e));              \
  } while (0)

#define TM_CHECK_MESH(ctx)                                                                  \
  do {                                                                                      \
    if (!(ctx)->has_mesh) return fail(ctx, TM_ESTATE, "no mesh uploaded");                  \
  } while (0)

template <typename T>
cudaError_t upload(std::vector<void *> &owned, int64_t &bytes, T **dst, const std::vector<T> &src) {
  const size_t n = std::max<size_t>(src.size(), 1);
  cudaError_t e = cudaMalloc((void **)dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  owned.push_back(*dst);
  bytes += (int64_t)(n * sizeof(T));
  if (!src.empty()) return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return cudaSuccess;
}

template <typename T>
cudaError_t alloc(std::vector<void *> &owned, int64_t &bytes, T **dst, size_t n) {
  n = std::max<size_t>(n, 1);
  cudaError_t e = cudaMalloc((void **)dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  owned.push_back(*dst);
  bytes += (int64_t)(n * sizeof(T));
  return cudaMemset(*dst, 0, n * sizeof(T));
}

void release(std::vector<void *> &owned) {
  for (void *p : owned) cudaFree(p);
  owned.clear();
}

// Scalars region layout (doubles): [0, 64) SolveScalars, [64, 80) OcState, [80] compliance,
// [81] outer rr, [82] ff, [90, 92) the two sums of the design difference (Eq. 10), [92] the load
// scale of the learned guess's input.
// Last-CTA tickets (w.ticket[16]): 0 CG update, 1 FP64 residual, 2 CG start / residual
// replacement, 3 sensitivity, 4 OC, 5 operator block pass, 6 design difference,
// 7 multi-vector block pass, 8 two-level CG scalars, 9 load scale of the learned guess.  Kernels that share a ticket never run
// concurrently (one stream).
constexpr int kScalDoubles = 128;
SolveScalars *solve_scalars(tm_ctx *c) { return reinterpret_cast<SolveScalars *>(c->w.scal); }
static_assert(sizeof(OcState) <= 16 * sizeof(double), "the OC state must end before scalar 80");
OcState *oc_state(tm_ctx *c) { return reinterpret_cast<OcState *>(c->w.scal + 64); }
double *scal_at(tm_ctx *c, int i) { return c->w.scal + i; }

// Event record on the context's stream; while a graph is being captured the
// record becomes a node of the graph (re-recorded at every replay).
cudaError_t record_event(tm_ctx *ctx, cudaEvent_t e) {
  if (ctx->capturing) return cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal);
  return cudaEventRecord(e, ctx->stream);
}

// Operator launches with optional CUDA-event timing (tm_profile): each timed
// application records an event pair on the context's stream; pairs are read
// back at the next synchronisation point.
template <typename T>
int timed_apply(tm_ctx *ctx, const T *ce, const T *x, T *y, T *part, double *dotp, SolveScalars *sc,
                bool zero_hanging, const int *done) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->prof_on) {
    if (ctx->ev_free.size() < 2) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        TM_CUDA(ctx, cudaEventCreate(&e));
        ctx->ev_free.push_back(e);
      }
    }
    e0 = ctx->ev_free.back(); ctx->ev_free.pop_back();
    e1 = ctx->ev_free.back(); ctx->ev_free.pop_back();
    TM_CUDA(ctx, record_event(ctx, e0));
  }
  TM_CUDA(ctx, launch_apply<T>(ctx->dm, ce, x, y, part, dotp, sc, ctx->w.ticket + 5, zero_hanging, done, ctx->stream));
  ctx->launches += 2;
  if (ctx->prof_on) {
    TM_CUDA(ctx, record_event(ctx, e1));
    ctx->ev_pending.push_back({e0, e1, sizeof(T) == 4 ? 1 : 0, false});
  }
  return TM_OK;
}

// The block pass alone (CG iterations): shared nodes stay in their partials.
template <typename T>
int timed_apply_blocks(tm_ctx *ctx, const T *ce, const T *x, T *y, T *part, double *energy_partials,
                       SolveScalars *sc, const int *done) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->prof_on) {
    if (ctx->ev_free.size() < 2) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        TM_CUDA(ctx, cudaEventCreate(&e));
        ctx->ev_free.push_back(e);
      }
    }
    e0 = ctx->ev_free.back(); ctx->ev_free.pop_back();
    e1 = ctx->ev_free.back(); ctx->ev_free.pop_back();
    TM_CUDA(ctx, record_event(ctx, e0));
  }
  TM_CUDA(ctx, launch_apply_blocks<T>(ctx->dm, ce, x, y, part, energy_partials, sc, ctx->w.ticket + 5, done,
                                      ctx->stream));
  ctx->launches += 1;
  if (ctx->prof_on) {
    TM_CUDA(ctx, record_event(ctx, e1));
    ctx->ev_pending.push_back({e0, e1, sizeof(T) == 4 ? 1 : 0, false});
  }
  return TM_OK;
}

// Accumulate completed event pairs (all of them when `all`, after a sync).
int drain_profile(tm_ctx *ctx, bool all) {
  std::vector<tm_ctx::Pending> keep;
  for (const auto &pe : ctx->ev_pending) {
    if (!all && cudaEventQuery(pe.e1) != cudaSuccess) {
      keep.push_back(pe);
      continue;
    }
    float ms = 0;
    TM_CUDA(ctx, cudaEventElapsedTime(&ms, pe.e0, pe.e1));
    // an apply skipped by the device-side done flag is not a launch that did work
    if (pe.kind == 1) { ctx->prof.apply32_ms += ms; ctx->prof.apply32_count++; }
    else { ctx->prof.apply64_ms += ms; ctx->prof.apply64_count++; }
    if (!pe.graph_owned) {
      ctx->ev_free.push_back(pe.e0);
      ctx->ev_free.push_back(pe.e1);
    }
  }
  ctx->ev_pending.swap(keep);
  return TM_OK;
}

void drop_graphs(tm_ctx *ctx) {
  for (auto &g : ctx->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto &pe : g.ev) {
      cudaEventDestroy(pe.e0);
      cudaEventDestroy(pe.e1);
    }
  }
  ctx->graphs.clear();
}

int read_scalar(tm_ctx *ctx, const double *dev, double *out) {
  TM_CUDA(ctx, cudaMemcpyAsync(out, dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TM_OK;
}

// f = C^T f_full for a few point loads: a load on a hanging node goes to its
// masters with the interpolation weights; loads on Dirichlet DOFs vanish.  One
// thread walks the loads in order (deterministic; loads are few).
__global__ void scatter_loads_kernel(const int64_t *idx, const double *val, int64_t n, const uint8_t *nflag,
                                     const int32_t *hang_node, const int32_t *hang_master, int64_t nh, double *f) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t node = idx[i] / 3;
    const int c = (int)(idx[i] % 3);
    if (nflag[node] & 2) {
      int64_t lo = 0, hi = nh - 1;
      while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (hang_node[mid] < node) lo = mid + 1;
        else hi = mid;
      }
      const int nm = hang_master[4 * lo + 2] < 0 ? 2 : 4;
      const double w = nm == 2 ? 0.5 : 0.25;
      for (int q = 0; q < nm; ++q) {
        const int mm = hang_master[4 * lo + q];
        if (!(nflag[mm] & 1)) f[3 * (int64_t)mm + c] += w * val[i];
      }
    } else if (!(nflag[node] & 1)) {
      f[idx[i]] += val[i];
    }
  }
}

void release_coarse(tm_ctx *ctx) {
  release(ctx->coarse.owned);
  ctx->coarse = CoarseHierarchy();
  ctx->coarse_ready = false;
}

void release_learn(tm_ctx *ctx) {
  release(ctx->learn.owned);
  ctx->learn = LearnTables();
}

// Voxel grid of level g and its tables for the uploaded mesh (first use, or another g).
int ensure_learn(tm_ctx *ctx, int g) {
  const HostMesh &hm = ctx->host;
  if (g < 0 || g > hm.L) return fail(ctx, TM_EINVAL, "voxel level g must be in [0, max_level]");
  const int X = hm.nx << g, Y = hm.ny << g, Z = hm.nz << g;
  if (X < 2 || Y < 2 || Z < 2) return fail(ctx, TM_EINVAL, "the voxel grid needs at least 2 cells per axis");
  LearnTables &t = ctx->learn;
  if (t.g == g) return TM_OK;
  release_learn(ctx);
  const int hv = 1 << (hm.L - g);
  std::vector<int32_t> cnt((size_t)X * Y * Z + 1, 0), anchor(hm.Nn);
  auto lower = [](int p, int n, int h) {
    const int i = (int)std::floor((double)p / h - 0.5);
    return i < 0 ? 0 : (i > n - 2 ? n - 2 : i);
  };
  for (int64_t n = 0; n < hm.Nn; ++n) {
    const int32_t *p = &hm.node_xyz[3 * n];
    const int a = (lower(p[0], X, hv) * Y + lower(p[1], Y, hv)) * Z + lower(p[2], Z, hv);
    anchor[n] = a;
    cnt[a + 1]++;
  }
  for (size_t i = 1; i < cnt.size(); ++i) cnt[i] += cnt[i - 1];
  std::vector<int32_t> vnode(hm.Nn), fill(cnt.begin(), cnt.end() - 1);
  for (int64_t n = 0; n < hm.Nn; ++n) vnode[fill[anchor[n]]++] = (int32_t)n;
  TM_CUDA(ctx, upload(t.owned, t.bytes, &t.nxyz, hm.node_xyz));
  TM_CUDA(ctx, upload(t.owned, t.bytes, &t.vptr, cnt));
  TM_CUDA(ctx, upload(t.owned, t.bytes, &t.vnode, vnode));
  TM_CUDA(ctx, alloc(t.owned, t.bytes, &t.pf, 3 * (size_t)X * Y * Z));
  t.g = g; t.X = X; t.Y = Y; t.Z = Z; t.hv = hv;
  return TM_OK;
}

// Tables and buffers of the two-level preconditioner for the uploaded mesh (first use).
int ensure_coarse(tm_ctx *ctx) {
  CoarseHierarchy &h = ctx->coarse;
  if (h.nlev > 0) return TM_OK;
  const HostMesh &hm = ctx->host;
  std::vector<int> shapes;
  std::string msg = coarse_shapes(hm, shapes);
  if (!msg.empty()) return fail(ctx, TM_EINVAL, "two-level preconditioner: " + msg);
  std::vector<int32_t> cell_elem, cptr, cnode, ncell;
  std::vector<uint32_t> code;
  std::vector<double> Q;
  coarse_tables(hm, cell_elem, cptr, cnode, ncell, code);
  std::vector<int32_t> seg_ptr, seg_cell, cseg;
  coarse_segments(cptr, seg_ptr, seg_cell, cseg);
  coarse_moment_matrices(hm.nu, Q);
  std::vector<void *> &o = h.owned;
  int64_t &B = h.bytes;
  TM_CUDA(ctx, upload(o, B, &h.cell_elem, cell_elem));
  TM_CUDA(ctx, upload(o, B, &h.cptr, cptr));
  TM_CUDA(ctx, upload(o, B, &h.cnode, cnode));
  TM_CUDA(ctx, upload(o, B, &h.ncell, ncell));
  TM_CUDA(ctx, upload(o, B, &h.code, code));
  {
    std::vector<uint32_t> ccode(cnode.size());   // the codes in cnode order
    for (size_t p = 0; p < cnode.size(); ++p) ccode[p] = code[cnode[p]];
    TM_CUDA(ctx, upload(o, B, &h.ccode, ccode));
  }
  TM_CUDA(ctx, upload(o, B, &h.seg_ptr, seg_ptr));
  TM_CUDA(ctx, upload(o, B, &h.seg_cell, seg_cell));
  TM_CUDA(ctx, upload(o, B, &h.cseg, cseg));
  h.nseg = (int32_t)seg_cell.size();
  {
    // the symmetric cell matrices by upper-triangle entry, with the moments that contribute
    std::vector<int32_t> qent(kCellUpper);
    std::vector<uint8_t> qidx((size_t)kCellUpper * kCellNnz, 0);
    std::vector<double> qval((size_t)kCellUpper * kCellNnz, 0.0);
    int u = 0;
    for (int i = 0; i < 24; ++i)
      for (int j = i; j < 24; ++j, ++u) {
        int nnz = 0;
        for (int q = 0; q < 27; ++q) {
          const double v = Q[(size_t)q * 576 + 24 * i + j];
          if (v != 0.0) {
            qidx[(size_t)u * kCellNnz + nnz] = (uint8_t)q;
            qval[(size_t)u * kCellNnz + nnz] = v;
            ++nnz;
          }
        }
        qent[u] = i | (j << 5) | (nnz << 10);
      }
    TM_CUDA(ctx, upload(o, B, &h.qent, qent));
    TM_CUDA(ctx, upload(o, B, &h.qidx, qidx));
    TM_CUDA(ctx, upload(o, B, &h.qval, qval));
  }
  const int nlev = (int)shapes.size() / 3;
  for (int l = 0; l < nlev; ++l) {
    CoarseLevel &c = h.lev[l];
    c.X = shapes[3 * l]; c.Y = shapes[3 * l + 1]; c.Z = shapes[3 * l + 2];
    c.nodes = (c.X + 1) * (c.Y + 1) * (c.Z + 1);
    c.H = std::ldexp(hm.h0, l);
    const size_t cells = (size_t)c.X * c.Y * c.Z, n3 = 3 * (size_t)c.nodes;
    TM_CUDA(ctx, alloc(o, B, &c.mom, 27 * cells));
    TM_CUDA(ctx, alloc(o, B, &c.K, 576 * cells));
    TM_CUDA(ctx, alloc(o, B, &c.dinv, n3));
    TM_CUDA(ctx, alloc(o, B, &c.b, kMaxRhs * n3));
    TM_CUDA(ctx, alloc(o, B, &c.x, kMaxRhs * n3));
    TM_CUDA(ctx, alloc(o, B, &c.x2, kMaxRhs * n3));
    TM_CUDA(ctx, alloc(o, B, &c.t, kMaxRhs * n3));
  }
  const CoarseLevel &cl = h.lev[nlev - 1];
  const size_t nc = 3 * (size_t)cl.nodes;
  TM_CUDA(ctx, alloc(o, B, &h.Kc64, 576 * (size_t)cl.X * cl.Y * cl.Z));
  TM_CUDA(ctx, alloc(o, B, &h.Ainv, nc * nc));
  TM_CUDA(ctx, alloc(o, B, &h.part, kMaxRhs * 24 * (size_t)h.nseg));
  h.faces = hm.dirichlet_faces;
  h.nlev = nlev;
  return TM_OK;
}

// Level operators, smoother diagonals and the coarsest inverse for the density rho, in two
// halves: coarse_setup_begin enqueues the device part and the copy of the coarsest level's cell
// matrices to the host; coarse_setup_end inverts on the host and enqueues the inverse's upload.
// Work the caller enqueues in between (the solver's first true residual) runs on the GPU while
// the host inverts.  Host time of the two halves is added to *seconds (may be NULL).
int coarse_setup_begin(tm_ctx *ctx, const double *rho, double *seconds) {
  const auto t0 = std::chrono::steady_clock::now();
  int rc = ensure_coarse(ctx);
  if (rc) return rc;
  CoarseHierarchy &h = ctx->coarse;
  ctx->coarse_ready = false;
  TM_CUDA(ctx, coarse_setup_launch(ctx->dm, h, rho, ctx->stream));
  ctx->launches += 3 * (int64_t)h.nlev - 1;
  const CoarseLevel &cl = h.lev[h.nlev - 1];
  h.Kc_host.resize(576 * (size_t)cl.X * cl.Y * cl.Z);
  TM_CUDA(ctx, cudaMemcpyAsync(h.Kc_host.data(), h.Kc64, h.Kc_host.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               ctx->stream));
  TM_CUDA(ctx, cudaEventRecord(ctx->ev_coarse, ctx->stream));
  if (seconds) *seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return TM_OK;
}

int coarse_setup_end(tm_ctx *ctx, double *seconds) {
  const auto t0 = std::chrono::steady_clock::now();
  CoarseHierarchy &h = ctx->coarse;
  const CoarseLevel &cl = h.lev[h.nlev - 1];
  TM_CUDA(ctx, cudaEventSynchronize(ctx->ev_coarse));   // the cell matrices are on the host
  std::vector<float> &Ainv = h.Ainv_host;
  std::string msg = coarse_dense_inverse(h.Kc_host, cl.X, cl.Y, cl.Z, h.faces, Ainv);
  if (!msg.empty()) return fail(ctx, TM_ENONFINITE, "two-level preconditioner: " + msg);
  TM_CUDA(ctx, cudaMemcpyAsync(h.Ainv, Ainv.data(), Ainv.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  ctx->coarse_ready = true;
  if (seconds) *seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return TM_OK;
}

int coarse_setup(tm_ctx *ctx, const double *rho, double *seconds) {
  if (seconds) *seconds = 0.0;
  int rc = coarse_setup_begin(ctx, rho, seconds);
  if (rc) return rc;
  rc = coarse_setup_end(ctx, seconds);
  if (rc) return rc;
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TM_OK;
}

// The two-level part of one preconditioner application on FP32 residuals: P0^T r, the V-cycle,
// the CG scalars (mode: 0 iteration, 1 start, 2 residual replacement; finish_kernel) and the
// search directions p from z = D^-1 r + P0 V(P0^T r), for load cases c0 .. c0 + nv - 1 (fine
// vectors ld apart, scalars sc[case], finish partials pstride apart, tickets[case]).
int enqueue_twolevel_cases(tm_ctx *ctx, int mode, const float *r, float *p, int64_t ld, const float *dinv, int nu,
                           SolveScalars *sc, int c0, int nv, double *partials, int pstride, unsigned int *tickets) {
  const CoarseHierarchy &h = ctx->coarse;
  TM_CUDA(ctx, coarse_restrict_launch(ctx->dm, h, r, ld, true, sc, c0, nv, ctx->stream));
  int nl = 0;
  TM_CUDA(ctx, coarse_vcycle_launch(h, nu, sc, c0, nv, ctx->stream, &nl));
  TM_CUDA(ctx, coarse_finish_launch(h, mode, sc, c0, nv, partials, pstride, tickets, ctx->stream));
  TM_CUDA(ctx, coarse_pupdate_launch(ctx->dm, h, p, r, ld, dinv, mode, sc, c0, nv, ctx->stream));
  ctx->launches += 4 + nl;
  return TM_OK;
}

// One load case on the context's single-solve vectors and scalars.
int enqueue_twolevel(tm_ctx *ctx, int mode, const float *r, float *p, const float *dinv, int nu) {
  return enqueue_twolevel_cases(ctx, mode, r, p, 3 * ctx->dm.Nn, dinv, nu, solve_scalars(ctx), 0, 1, ctx->w.red,
                                4 * device_sms(), ctx->w.ticket + 8);
}

}  // namespace

extern "C" {

int tm_create(tm_ctx **out, int device, void *cuda_stream) try {
  if (!out) return TM_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) return TM_ECUDA;
  if (device < 0 || device >= n) return TM_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return TM_ECUDA;
  tm_ctx *c = new tm_ctx();
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_coarse, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return TM_ECUDA;
  }
  *out = c;
  return TM_OK;
} catch (...) {
  return exception_status(nullptr);
}

int tm_destroy(tm_ctx *ctx) try {
  if (!ctx) return TM_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaStreamSynchronize(ctx->gstream);
  drop_graphs(ctx);
  release_coarse(ctx);
  release_learn(ctx);
  release(ctx->dm.owned);
  release(ctx->w.owned);
  for (auto &pe : ctx->ev_pending) {
    cudaEventDestroy(pe.e0);
    cudaEventDestroy(pe.e1);
  }
  for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_coarse) cudaEventDestroy(ctx->ev_coarse);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  delete ctx;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_set_stream(tm_ctx *ctx, void *cuda_stream) try {
  if (!ctx) return TM_EINVAL;
  ctx->stream = (cudaStream_t)cuda_stream;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

const char *tm_last_error(tm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tm_mesh_upload(tm_ctx *ctx, const tm_mesh_desc *d, tm_mesh_info *info) try {
  TM_CHECK_CTX(ctx);
  if (!d) return fail(ctx, TM_EINVAL, "null mesh descriptor");
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  drop_graphs(ctx);
  ctx->has_mesh = false;
  release_coarse(ctx);
  release_learn(ctx);
  release(ctx->dm.owned);
  release(ctx->w.owned);
  ctx->dm = DeviceMesh();
  ctx->w = Work();
  HostMesh &h = ctx->host;
  std::string msg = build_host_mesh(*d, h);
  if (!msg.empty()) return fail(ctx, TM_EINVAL, msg);

  DeviceMesh &m = ctx->dm;
  m.Ne = h.Ne; m.Nn = h.Nn; m.nh = (int64_t)h.hang_node.size(); m.nsh = (int64_t)h.sh_node.size();
  m.nblk = h.nblk; m.L = h.L; m.max_local = h.max_local;
  m.fx = h.nx << h.L; m.fy = h.ny << h.L; m.fz = h.nz << h.L;
  m.h0 = h.h0; m.hmin = std::ldexp(h.h0, -h.L);
  m.E0 = h.E0; m.Emin = h.Emin; m.penal = h.penal; m.nu = h.nu;
  for (int i = 0; i < 72; ++i) m.modal[i] = h.modal[i];
  m.k0diag = h.K0[0];
  m.volume = (double)h.nx * h.ny * h.nz * h.h0 * h.h0 * h.h0;
  m.n_free = 3 * h.n_free_nodes;
  m.nslot = h.nslot;
  m.nbrick = h.nbrick;
  std::vector<void *> &o = m.owned;
  int64_t &B = m.bytes;
  TM_CUDA(ctx, upload(o, B, &m.leaf, h.leaf));
  TM_CUDA(ctx, upload(o, B, &m.cellmap, h.cellmap));
  TM_CUDA(ctx, upload(o, B, &m.conn, h.conn));
  TM_CUDA(ctx, upload(o, B, &m.nflag, h.nflag));
  TM_CUDA(ctx, upload(o, B, &m.hang_node, h.hang_node));
  TM_CUDA(ctx, upload(o, B, &m.hang_master, h.hang_master));
  TM_CUDA(ctx, upload(o, B, &m.blk_elem, h.blk_elem));
  TM_CUDA(ctx, upload(o, B, &m.blk_node, h.blk_node));
  TM_CUDA(ctx, upload(o, B, &m.blk_shared, h.blk_shared));
  TM_CUDA(ctx, upload(o, B, &m.blk_slot, h.blk_slot));
  TM_CUDA(ctx, upload(o, B, &m.blk_hang, h.blk_hang));
  TM_CUDA(ctx, upload(o, B, &m.blk_iptr, h.blk_iptr));
  TM_CUDA(ctx, upload(o, B, &m.blk_inv, h.blk_inv));
  TM_CUDA(ctx, upload(o, B, &m.lnode, h.lnode));
  TM_CUDA(ctx, upload(o, B, &m.lslot, h.lslot));
  TM_CUDA(ctx, upload(o, B, &m.hent, h.hent));
  TM_CUDA(ctx, upload(o, B, &m.iptr, h.iptr));
  TM_CUDA(ctx, upload(o, B, &m.inv, h.inv));
  {
    uint8_t *rec = nullptr;
    TM_CUDA(ctx, upload(o, B, &rec, h.brec));
    m.brec = reinterpret_cast<uint4 *>(rec);
  }
  TM_CUDA(ctx, upload(o, B, &m.rec_off, h.rec_off));
  TM_CUDA(ctx, upload(o, B, &m.rec_skip, h.rec_skip));
  m.max_rec_bytes = h.max_rec_bytes;
  m.max_rec_stage = h.max_rec_stage;
  TM_CUDA(ctx, upload(o, B, &m.brick_tab, h.brick_tab));
  TM_CUDA(ctx, apply_residency(m, &m.resident_cta32, &m.resident_cta64));
  TM_CUDA(ctx, upload(o, B, &m.sh_node, h.sh_node));
  TM_CUDA(ctx, upload(o, B, &m.sh_ptr, h.sh_ptr));
  TM_CUDA(ctx, upload(o, B, &m.sh_of_node, h.sh_of_node));
  TM_CUDA(ctx, upload(o, B, &m.dg_ptr, h.dg_ptr));
  TM_CUDA(ctx, upload(o, B, &m.dg_elem, h.dg_elem));
  TM_CUDA(ctx, upload(o, B, &m.dg_q, h.dg_q));
  TM_CUDA(ctx, upload(o, B, &m.dg_tab, h.dg_tab));
  // the host keeps only what tm_mesh_tables / tm_build_rhs need
  std::vector<int32_t>().swap(h.cellmap);
  std::vector<int32_t>().swap(h.dg_elem);
  std::vector<uint16_t>().swap(h.dg_q);
  std::vector<int32_t>().swap(h.dg_ptr);

  Work &w = ctx->w;
  std::vector<void *> &wo = w.owned;
  int64_t &WB = w.bytes;
  const size_t nv = 3 * (size_t)m.Nn;
  w.nred = (int64_t)apply_ctas(m) + (m.nsh + m.nh + 255) / 256 + 8 * 8 * (int64_t)device_sms() + 64;
  TM_CUDA(ctx, alloc(wo, WB, &w.part64, 3 * (size_t)m.nslot));
  TM_CUDA(ctx, alloc(wo, WB, &w.part32, 3 * (size_t)m.nslot));
  TM_CUDA(ctx, alloc(wo, WB, &w.ce64, (size_t)m.Ne));
  TM_CUDA(ctx, alloc(wo, WB, &w.ce32, (size_t)m.Ne));
  TM_CUDA(ctx, alloc(wo, WB, &w.red, (size_t)w.nred));
  TM_CUDA(ctx, alloc(wo, WB, &w.scal, (size_t)kScalDoubles));
  TM_CUDA(ctx, alloc(wo, WB, &w.ticket, (size_t)16));
  TM_CUDA(ctx, alloc(wo, WB, &w.status, (size_t)16));
  TM_CUDA(ctx, alloc(wo, WB, &w.mark_tmp, (size_t)m.Ne));
  TM_CUDA(ctx, alloc(wo, WB, &w.r, nv));
  TM_CUDA(ctx, alloc(wo, WB, &w.p, nv));
  TM_CUDA(ctx, alloc(wo, WB, &w.q, nv));
  TM_CUDA(ctx, alloc(wo, WB, &w.dinv, nv));
  TM_CUDA(ctx, alloc(wo, WB, &w.r32, nv));
  TM_CUDA(ctx, alloc(wo, WB, &w.p32, nv));
  TM_CUDA(ctx, alloc(wo, WB, &w.q32, nv));
  TM_CUDA(ctx, alloc(wo, WB, &w.dinv32, nv));
  TM_CUDA(ctx, alloc(wo, WB, &w.x32, nv));
  TM_CUDA(ctx, cudaDeviceSynchronize());
  ctx->has_mesh = true;
  if (info) {
    info->Ne = m.Ne;
    info->Nn = m.Nn;
    info->n_hanging = m.nh;
    info->n_dirichlet = h.n_dirichlet;
    info->n_free = m.n_free;
    info->n_blocks = m.nblk;
    info->max_local = h.max_local;
    info->n_shared = m.nsh;
    info->device_bytes = m.bytes + w.bytes;
    info->max_block_bytes = h.max_rec_bytes;
    info->n_bricks = m.nbrick;
  }
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_mesh_tables(tm_ctx *ctx, int64_t *perm, int32_t *node_xyz, int32_t *conn, int32_t *hang_node,
                   int32_t *hang_master, uint8_t *node_flags) try {
  if (!ctx) return TM_EINVAL;
  TM_CHECK_MESH(ctx);
  const HostMesh &h = ctx->host;
  if (perm) std::memcpy(perm, h.perm.data(), h.perm.size() * sizeof(int64_t));
  if (node_xyz) std::memcpy(node_xyz, h.node_xyz.data(), h.node_xyz.size() * sizeof(int32_t));
  if (conn) std::memcpy(conn, h.conn.data(), h.conn.size() * sizeof(int32_t));
  if (hang_node) std::memcpy(hang_node, h.hang_node.data(), h.hang_node.size() * sizeof(int32_t));
  if (hang_master) std::memcpy(hang_master, h.hang_master.data(), h.hang_master.size() * sizeof(int32_t));
  if (node_flags) std::memcpy(node_flags, h.nflag.data(), h.nflag.size());
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_build_rhs(tm_ctx *ctx, int64_t n_loads, const int32_t *node_xyz, const int32_t *comp, const double *val,
                 double *f_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (n_loads < 0 || (n_loads > 0 && (!node_xyz || !comp || !val)) || !f_dev)
    return fail(ctx, TM_EINVAL, "bad load arguments");
  const HostMesh &h = ctx->host;
  std::vector<int64_t> idx(n_loads);
  for (int64_t i = 0; i < n_loads; ++i) {
    const int32_t x = node_xyz[3 * i], y = node_xyz[3 * i + 1], z = node_xyz[3 * i + 2];
    if (x < 0 || y < 0 || z < 0 || comp[i] < 0 || comp[i] > 2) return fail(ctx, TM_EINVAL, "bad load");
    const uint64_t k = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
    auto it = std::lower_bound(h.node_key.begin(), h.node_key.end(), k);
    if (it == h.node_key.end() || *it != k) return fail(ctx, TM_EINVAL, "load point is not a mesh node");
    idx[i] = 3 * (int64_t)(it - h.node_key.begin()) + comp[i];
  }
  const DeviceMesh &m = ctx->dm;
  TM_CUDA(ctx, cudaMemsetAsync(f_dev, 0, 3 * (size_t)m.Nn * sizeof(double), ctx->stream));
  if (n_loads > 0) {
    int64_t *didx = nullptr;
    double *dval = nullptr;
    TM_CUDA(ctx, cudaMalloc(&didx, n_loads * sizeof(int64_t)));
    cudaError_t e = cudaMalloc(&dval, n_loads * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(didx, idx.data(), n_loads * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dval, val, n_loads * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
      scatter_loads_kernel<<<1, 32, 0, ctx->stream>>>(didx, dval, n_loads, m.nflag, m.hang_node, m.hang_master,
                                                       m.nh, f_dev);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(didx);
    cudaFree(dval);
    TM_CUDA(ctx, e);
  }
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_apply_K(tm_ctx *ctx, const double *rho_dev, const double *x_dev, double *y_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !x_dev || !y_dev) return fail(ctx, TM_EINVAL, "null pointer");
  TM_CUDA(ctx, launch_coeff(ctx->dm, ctx->w, rho_dev, ctx->stream));
  ctx->launches += 1;
  int rc = timed_apply<double>(ctx, ctx->w.ce64, x_dev, y_dev, ctx->w.part64, nullptr, nullptr, true, nullptr);
  if (rc) return rc;
  return drain_profile(ctx, false);
} catch (...) {
  return exception_status(ctx);
}

int tm_apply_K_f32(tm_ctx *ctx, const double *rho_dev, const float *x_dev, float *y_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !x_dev || !y_dev) return fail(ctx, TM_EINVAL, "null pointer");
  TM_CUDA(ctx, launch_coeff(ctx->dm, ctx->w, rho_dev, ctx->stream));
  ctx->launches += 1;
  int rc = timed_apply<float>(ctx, ctx->w.ce32, x_dev, y_dev, ctx->w.part32, nullptr, nullptr, true, nullptr);
  if (rc) return rc;
  return drain_profile(ctx, false);
} catch (...) {
  return exception_status(ctx);
}

int tm_apply_K_f32_multi(tm_ctx *ctx, int nrhs, const double *rho_dev, const float *x_dev, float *y_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !x_dev || !y_dev) return fail(ctx, TM_EINVAL, "null pointer");
  if (nrhs < 1 || nrhs > kMaxRhs) return fail(ctx, TM_EINVAL, "nrhs must be in [1, " + std::to_string(kMaxRhs) + "]");
  Work &w = ctx->w;
  if (!w.part_multi) TM_CUDA(ctx, alloc(w.owned, w.bytes, &w.part_multi, (size_t)kMaxRhs * 3 * ctx->dm.nslot));
  TM_CUDA(ctx, launch_coeff_f32(ctx->dm, rho_dev, w.ce32, ctx->stream));
  TM_CUDA(ctx, launch_apply_multi(ctx->dm, nrhs, w.ce32, x_dev, y_dev, w.part_multi, nullptr, nullptr, nullptr,
                                  ctx->stream));
  ctx->launches += 3;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_apply_K_f32_static(tm_ctx *ctx, const double *rho_dev, const float *x_dev, float *y_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !x_dev || !y_dev) return fail(ctx, TM_EINVAL, "null pointer");
  const DeviceMesh &m = ctx->dm;
  if (m.Ne > kStaticElems || m.nslot > kStaticSlots)
    return fail(ctx, TM_EINVAL,
                "mesh too large for the static scratch of tm_apply_K_f32_static: " + std::to_string(m.Ne) +
                    " elements (max " + std::to_string(kStaticElems) + "), " + std::to_string(m.nslot) +
                    " shared-node partials (max " + std::to_string(kStaticSlots) + ")");
  float *ce = nullptr, *part = nullptr;
  TM_CUDA(ctx, static_scratch(ctx->device, &ce, &part));
  TM_CUDA(ctx, launch_coeff_f32(m, rho_dev, ce, ctx->stream));
  TM_CUDA(ctx, launch_apply<float>(m, ce, x_dev, y_dev, part, nullptr, nullptr, nullptr, true, nullptr, ctx->stream));
  ctx->launches += 3;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_jacobi_diag(tm_ctx *ctx, const double *rho_dev, double *d_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !d_dev) return fail(ctx, TM_EINVAL, "null pointer");
  TM_CUDA(ctx, launch_coeff(ctx->dm, ctx->w, rho_dev, ctx->stream));
  TM_CUDA(ctx, launch_diag(ctx->dm, ctx->w.ce64, d_dev, nullptr, nullptr, ctx->stream));
  ctx->launches += 2;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_pcg_solve_batch(int n, tm_ctx *const *ctxs, const double *const *rho_dev, const double *const *f_dev,
                       double *const *u_dev, const tm_solve_opts *opts, tm_solve_stats *stats, int *status) try {
  if (n < 1 || !ctxs || !rho_dev || !f_dev || !u_dev || !opts) return TM_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return TM_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(ctxs[i], TM_EINVAL, "a context appears twice in one batch");
  }
  // one host thread per context: each drives its own solve on its own streams, so the
  // solves' kernels, graph replays and convergence checks interleave on the GPU
  // (a solve whose thread cannot be started runs on the calling thread)
  std::vector<int> rc(n, TM_OK);
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i) {
    auto solve = [&, i] {
      rc[i] = tm_pcg_solve(ctxs[i], rho_dev[i], f_dev[i], u_dev[i], opts, stats ? &stats[i] : nullptr);
    };
    try {
      th.emplace_back(solve);
    } catch (...) {
      solve();
    }
  }
  for (auto &t : th) t.join();
  int first = TM_OK;
  for (int i = 0; i < n; ++i) {
    if (status) status[i] = rc[i];
    if (first == TM_OK && rc[i] != TM_OK) first = rc[i];
  }
  return first;
} catch (...) {
  return exception_status(nullptr);
}

int tm_expand(tm_ctx *ctx, const double *u_dev, double *u_full_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!u_dev || !u_full_dev) return fail(ctx, TM_EINVAL, "null pointer");
  TM_CUDA(ctx, launch_expand(ctx->dm, u_dev, u_full_dev, ctx->stream));
  ctx->launches += ctx->dm.nh > 0 ? 2 : 1;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_amr_mark(tm_ctx *ctx, const double *rho_dev, double rho_solid, double r_amr, int8_t *mark_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !mark_dev) return fail(ctx, TM_EINVAL, "null pointer");
  if (!(r_amr >= 0) || r_amr > 4.0 * ctx->dm.hmin) return fail(ctx, TM_EINVAL, "r_amr must be in [0, 4 h_min]");
  TM_CUDA(ctx, launch_amr_mark(ctx->dm, rho_dev, rho_solid, r_amr, ctx->w.mark_tmp, mark_dev, ctx->stream));
  ctx->launches += 3;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_amr_adapt(tm_ctx *ctx, const int8_t *mark_dev, const double *rho_dev, int64_t capacity, int32_t *leaves_out,
                 double *rho_out, int64_t *n_out) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!mark_dev || !rho_dev || !n_out) return fail(ctx, TM_EINVAL, "null pointer");
  const int64_t Ne = ctx->dm.Ne;
  std::vector<int8_t> mk(Ne);
  std::vector<double> r(Ne);
  TM_CUDA(ctx, cudaMemcpyAsync(mk.data(), mark_dev, Ne, cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaMemcpyAsync(r.data(), rho_dev, Ne * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<int32_t> lv;
  std::vector<double> rn;
  std::string msg = adapt_leaves(ctx->host, mk.data(), r.data(), lv, rn);
  if (!msg.empty()) return fail(ctx, TM_EINVAL, msg);
  *n_out = (int64_t)rn.size();
  if ((int64_t)rn.size() > capacity || !leaves_out || !rho_out)
    return fail(ctx, TM_EINVAL, "capacity " + std::to_string(capacity) + " < " + std::to_string(rn.size()) + " leaves");
  std::memcpy(leaves_out, lv.data(), lv.size() * sizeof(int32_t));
  std::memcpy(rho_out, rn.data(), rn.size() * sizeof(double));
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_design_difference(tm_ctx *ctx, const double *rho_dev, int64_t n_other, const int32_t *leaves_other,
                         const double *rho_other, double *d_out) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !leaves_other || !rho_other || !d_out || n_other < 1) return fail(ctx, TM_EINVAL, "bad arguments");
  const HostMesh &h = ctx->host;
  {
    // the other design must tile the same box with leaves of levels 0..L, each cell once
    const int64_t ext[3] = {(int64_t)h.nx << h.L, (int64_t)h.ny << h.L, (int64_t)h.nz << h.L};
    std::vector<uint8_t> seen((size_t)(ext[0] * ext[1] * ext[2]), 0);
    int64_t covered = 0;
    for (int64_t i = 0; i < n_other; ++i) {
      const int32_t *l = leaves_other + 4 * i;
      if (l[3] < 0 || l[3] > h.L) return fail(ctx, TM_EINVAL, "other design: leaf level out of range");
      const int64_t s = (int64_t)1 << (h.L - l[3]);
      for (int a = 0; a < 3; ++a)
        if (l[a] < 0 || l[a] + s > ext[a] || l[a] % s) return fail(ctx, TM_EINVAL, "other design: misplaced leaf");
      for (int64_t z = l[2]; z < l[2] + s; ++z)
        for (int64_t y = l[1]; y < l[1] + s; ++y)
          for (int64_t x = l[0]; x < l[0] + s; ++x) {
            uint8_t &c = seen[(size_t)((z * ext[1] + y) * ext[0] + x)];
            if (c) return fail(ctx, TM_EINVAL, "other design: overlapping leaves");
            c = 1;
          }
      covered += s * s * s;
    }
    if (covered != (int64_t)seen.size()) return fail(ctx, TM_EINVAL, "other design does not cover the box");
  }
  const int64_t ncell = (int64_t)ctx->dm.fx * ctx->dm.fy * ctx->dm.fz;
  int32_t *dl = nullptr, *map2 = nullptr;
  double *dr = nullptr;
  cudaError_t e = cudaMalloc(&dl, n_other * 4 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&dr, n_other * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&map2, ncell * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(map2, 0xFF, ncell * sizeof(int32_t), ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dl, leaves_other, n_other * 4 * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dr, rho_other, n_other * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = launch_design_difference(ctx->dm, rho_dev, dl, n_other, dr, map2, ctx->w.red, ctx->w.ticket + 6, scal_at(ctx, 90),
                                 ctx->stream);
  double out[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, scal_at(ctx, 90), 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(dl);
  cudaFree(dr);
  cudaFree(map2);
  TM_CUDA(ctx, e);
  ctx->launches += 2;
  *d_out = out[0] / out[1];
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_transfer_displacement(tm_ctx *ctx, const double *u_full_dev, int64_t n_points, const int32_t *points_dev,
                             double *out_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (n_points < 0 || !u_full_dev || (n_points > 0 && (!points_dev || !out_dev)))
    return fail(ctx, TM_EINVAL, "bad arguments");
  if (n_points == 0) return TM_OK;
  int *bad = ctx->w.status + 1;
  TM_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
  TM_CUDA(ctx, launch_transfer(ctx->dm, u_full_dev, points_dev, n_points, out_dev, bad, ctx->stream));
  ctx->launches += 1;
  int nbad = 0;
  TM_CUDA(ctx, cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (nbad) return fail(ctx, TM_EINVAL, std::to_string(nbad) + " transfer points outside the mesh's box");
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_learn_input(tm_ctx *ctx, const double *rho_dev, const double *f_dev, int g, float *x_dev, double *s_out) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !f_dev || !x_dev) return fail(ctx, TM_EINVAL, "null pointer");
  int rc = ensure_learn(ctx, g);
  if (rc) return rc;
  double *s_dev = scal_at(ctx, 92);
  TM_CUDA(ctx, learn_input_launch(ctx->dm, ctx->learn, rho_dev, f_dev, ctx->learn.pf, ctx->w.red, ctx->w.ticket + 9,
                                  s_dev, x_dev, ctx->stream));
  ctx->launches += 4;
  double s = 0;
  rc = read_scalar(ctx, s_dev, &s);
  if (rc) return rc;
  if (!(s > 0) || !std::isfinite(s)) return fail(ctx, TM_EINVAL, "the load restricts to zero on the voxel grid");
  if (s_out) *s_out = s;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_learn_guess(tm_ctx *ctx, const float *out_dev, double s, int g, double *u0_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!out_dev || !u0_dev) return fail(ctx, TM_EINVAL, "null pointer");
  int rc = ensure_learn(ctx, g);
  if (rc) return rc;
  TM_CUDA(ctx, learn_guess_launch(ctx->dm, ctx->learn, out_dev, s, u0_dev, ctx->stream));
  ctx->launches += 1;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_learn_output_grad(tm_ctx *ctx, const double *au0_dev, const double *f_dev, double s, int g, float *dout_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!au0_dev || !f_dev || !dout_dev) return fail(ctx, TM_EINVAL, "null pointer");
  int rc = ensure_learn(ctx, g);
  if (rc) return rc;
  TM_CUDA(ctx, learn_grad_launch(ctx->dm, ctx->learn, au0_dev, f_dev, s, ctx->learn.pf, dout_dev, ctx->stream));
  ctx->launches += 2;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_adam_step(tm_ctx *ctx, int64_t n, float *params_dev, const float *grads_dev, float *m_dev, float *v_dev,
                 int step, float lr, float beta1, float beta2, float eps) try {
  TM_CHECK_CTX(ctx);
  if (n < 0 || (n > 0 && (!params_dev || !grads_dev || !m_dev || !v_dev)) || step < 1 || !(lr > 0) ||
      !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return fail(ctx, TM_EINVAL, "bad Adam arguments");
  if (n == 0) return TM_OK;
  const float c1 = 1.f - std::pow(beta1, (float)step), c2 = 1.f - std::pow(beta2, (float)step);
  TM_CUDA(ctx, adam_launch(params_dev, grads_dev, m_dev, v_dev, n, lr, beta1, beta2, eps, c1, c2, ctx->stream));
  ctx->launches += 1;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_profile(tm_ctx *ctx, int enable) try {
  TM_CHECK_CTX(ctx);
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int rc = drain_profile(ctx, true);
  if (rc) return rc;
  ctx->prof_on = enable != 0;
  ctx->launches = 0;
  ctx->prof = tm_profile_data();
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_profile_read(tm_ctx *ctx, tm_profile_data *out) try {
  TM_CHECK_CTX(ctx);
  if (!out) return fail(ctx, TM_EINVAL, "null pointer");
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int rc = drain_profile(ctx, true);
  if (rc) return rc;
  *out = ctx->prof;
  out->launches = ctx->launches;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

}  // extern "C"

// ---------------------------------------------------------------- solver drivers
namespace {

int init_run(tm_ctx *ctx, double stop_ratio2, double stop_abs_rr, int max_it) {
  SolveScalars s;
  std::memset(&s, 0, sizeof(s));
  s.stop_ratio2 = stop_ratio2;
  s.stop_abs_rr = stop_abs_rr;
  s.max_it = max_it;
  TM_CUDA(ctx, cudaMemcpyAsync(solve_scalars(ctx), &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TM_OK;
}

int read_run(tm_ctx *ctx, SolveScalars *s) {
  TM_CUDA(ctx, cudaMemcpyAsync(s, solve_scalars(ctx), sizeof(*s), cudaMemcpyDeviceToHost, ctx->stream));
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return drain_profile(ctx, false);
}

// Enqueue `count` CG iterations on vectors of type T (operator coefficients ce,
// partials part), solution x of type TX.  Three launches per iteration with the Jacobi
// preconditioner; with the two-level one (FP32 only) the coarse step replaces the p update.
template <typename TX, typename T>
int enqueue_iterations(tm_ctx *ctx, int count, const T *ce, T *part, TX *x, T *r, T *p, T *q, const T *dinv,
                       int precond, int nu) {
  Work &w = ctx->w;
  SolveScalars *sc = solve_scalars(ctx);
  const int64_t n = 3 * ctx->dm.Nn;
  const DeviceMesh &m = ctx->dm;
  const bool twolevel = precond == TM_PRECOND_TWOLEVEL;
  for (int k = 0; k < count; ++k) {
    int rc = timed_apply_blocks<T>(ctx, ce, p, q, part, w.red, sc, &sc->done);
    if (rc) return rc;
    TM_CUDA(ctx, launch_update_nodes<TX, T>(x, p, q, r, dinv, m.Nn, m.sh_of_node, m.sh_ptr, part, sc, w.red,
                                            w.ticket, ctx->stream, twolevel));
    ctx->launches += 1;
    if constexpr (std::is_same<T, float>::value) {
      if (twolevel) {
        rc = enqueue_twolevel(ctx, 0, r, p, dinv, nu);
        if (rc) return rc;
        continue;
      }
    }
    TM_CUDA(ctx, launch_pupdate<T>(p, r, dinv, n, sc, ctx->stream));
    ctx->launches += 1;
  }
  return TM_OK;
}

// Return event pairs to the pool unless a captured graph owns them.
void recycle(tm_ctx *ctx, const tm_ctx::Pending &pe) {
  if (pe.graph_owned) return;
  ctx->ev_free.push_back(pe.e0);
  ctx->ev_free.push_back(pe.e1);
}

// A batch of `count` CG iterations as a CUDA graph on the context's own stream,
// captured once per (vector set, batch size, profiling) and replayed.
template <typename TX, typename T>
int batch_graph(tm_ctx *ctx, int count, const T *ce, T *part, TX *x, T *r, T *p, T *q, const T *dinv, int precond,
                int nu, tm_ctx::Graph **out) {
  const void *key[4] = {(const void *)x, (const void *)r, (const void *)ce, (const void *)part};
  for (auto &g : ctx->graphs)
    if (g.count == count && g.prof == ctx->prof_on && g.precond == precond && g.nu == nu &&
        std::memcmp(g.key, key, sizeof(key)) == 0) {
      *out = &g;
      return TM_OK;
    }
  if (ctx->graphs.size() >= 8) {   // bounded cache: drop the oldest
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->gstream));
    tm_ctx::Graph &old = ctx->graphs.front();
    if (old.exec) cudaGraphExecDestroy(old.exec);
    for (auto &pe : old.ev) {
      cudaEventDestroy(pe.e0);
      cudaEventDestroy(pe.e1);
    }
    ctx->graphs.pop_front();
  }
  if (ctx->prof_on) {   // no event creation while capturing
    while (ctx->ev_free.size() < 2 * (size_t)count + 2) {
      cudaEvent_t ev;
      TM_CUDA(ctx, cudaEventCreate(&ev));
      ctx->ev_free.push_back(ev);
    }
  }
  tm_ctx::Graph g;
  std::memcpy(g.key, key, sizeof(key));
  g.count = count;
  g.prof = ctx->prof_on;
  g.precond = precond;
  g.nu = nu;
  const int64_t launches0 = ctx->launches;
  cudaStream_t user = ctx->stream;
  ctx->stream = ctx->gstream;
  ctx->capturing = true;
  const size_t base = ctx->ev_pending.size();
  cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
  int rc = TM_OK;
  if (e == cudaSuccess) rc = enqueue_iterations<TX, T>(ctx, count, ce, part, x, r, p, q, dinv, precond, nu);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(ctx->gstream, &graph);
  ctx->capturing = false;
  ctx->stream = user;
  // the pairs recorded while capturing belong to the graph
  for (size_t i = base; i < ctx->ev_pending.size(); ++i) {
    g.ev.push_back(ctx->ev_pending[i]);
    g.ev.back().graph_owned = true;
  }
  ctx->ev_pending.resize(base);
  g.launches = (int)(ctx->launches - launches0);
  ctx->launches = launches0;    // counted at replay
  if (e != cudaSuccess || rc || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, TM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    if (rc) return rc;
    return fail(ctx, TM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e2));
  }
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(ctx, TM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  ctx->graphs.push_back(std::move(g));
  *out = &ctx->graphs.back();
  return TM_OK;
}

template <typename TX, typename T>
int run_cg(tm_ctx *ctx, int check_every, bool graphs, int *iters_out, int *nonfinite, const T *ce, T *part, TX *x,
           T *r, T *p, T *q, const T *dinv, int precond = TM_PRECOND_JACOBI, int nu = 1) {
  SolveScalars s;
  int rc = read_run(ctx, &s);
  if (rc) return rc;
  tm_ctx::Graph *g = nullptr;
  if (graphs) {
    rc = batch_graph<TX, T>(ctx, check_every, ce, part, x, r, p, q, dinv, precond, nu, &g);
    if (rc) return rc;
  }
  while (!s.done) {
    const int it_before = s.it;
    const size_t base = ctx->ev_pending.size();
    if (g) {
      // user stream -> own stream -> user stream
      TM_CUDA(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
      TM_CUDA(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->ev_fork, 0));
      TM_CUDA(ctx, cudaGraphLaunch(g->exec, ctx->gstream));
      TM_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->gstream));
      TM_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
      ctx->launches += g->launches;
      for (const auto &pe : g->ev) ctx->ev_pending.push_back(pe);
    } else {
      rc = enqueue_iterations<TX, T>(ctx, check_every, ce, part, x, r, p, q, dinv, precond, nu);
      if (rc) return rc;
    }
    TM_CUDA(ctx, cudaMemcpyAsync(&s, solve_scalars(ctx), sizeof(s), cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    // applications enqueued after convergence returned at once: not timed work
    const size_t real = base + (size_t)(s.it - it_before);
    while (ctx->ev_pending.size() > real) {
      recycle(ctx, ctx->ev_pending.back());
      ctx->ev_pending.pop_back();
    }
    rc = drain_profile(ctx, true);
    if (rc) return rc;
  }
  *iters_out = s.it;
  *nonfinite = s.nonfinite;
  return TM_OK;
}

}  // namespace

extern "C" {

int tm_pcg_solve(tm_ctx *ctx, const double *rho_dev, const double *f_dev, double *u_dev, const tm_solve_opts *opts,
                 tm_solve_stats *stats) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !f_dev || !u_dev || !opts) return fail(ctx, TM_EINVAL, "null pointer");
  if (!(opts->rtol > 0) || opts->max_iter < 1) return fail(ctx, TM_EINVAL, "need rtol > 0 and max_iter >= 1");
  if (opts->precision != TM_PREC_FP64 && opts->precision != TM_PREC_MIXED)
    return fail(ctx, TM_EINVAL, "unknown precision");
  if (opts->precond != TM_PRECOND_JACOBI && opts->precond != TM_PRECOND_TWOLEVEL)
    return fail(ctx, TM_EINVAL, "unknown preconditioner");
  if (opts->precond == TM_PRECOND_TWOLEVEL && opts->precision != TM_PREC_MIXED)
    return fail(ctx, TM_EINVAL, "the two-level preconditioner runs with TM_PREC_MIXED");
  const bool twolevel = opts->precond == TM_PRECOND_TWOLEVEL;
  const int nu = opts->smooth_sweeps > 0 ? opts->smooth_sweeps : 1;
  const DeviceMesh &m = ctx->dm;
  Work &w = ctx->w;
  cudaStream_t st = ctx->stream;
  const int64_t n = 3 * m.Nn;
  const int check = opts->check_every > 0 ? opts->check_every : 32;
  const bool graphs = opts->no_graphs == 0;
  tm_solve_stats out;
  std::memset(&out, 0, sizeof(out));

  TM_CUDA(ctx, cudaEventRecord(ctx->ev0, st));
  TM_CUDA(ctx, launch_coeff(m, w, rho_dev, st));
  TM_CUDA(ctx, launch_diag(m, w.ce64, nullptr, w.dinv, w.dinv32, st));
  TM_CUDA(ctx, launch_mask(m.nflag, u_dev, m.Nn, st));
  double *ff_dev = scal_at(ctx, 82), *rr_dev = scal_at(ctx, 81);
  TM_CUDA(ctx, launch_residual64(f_dev, nullptr, nullptr, n, ff_dev, w.red, w.ticket + 1, st));
  ctx->launches += 4;
  double ff = 0;
  int rc = read_scalar(ctx, ff_dev, &ff);
  if (rc) return rc;
  if (!std::isfinite(ff)) return fail(ctx, TM_ENONFINITE, "non-finite load vector");
  int status = TM_OK;
  if (ff == 0.0) {
    TM_CUDA(ctx, cudaMemsetAsync(u_dev, 0, n * sizeof(double), st));
    out.rel_residual = 0.0;
  } else if (opts->precision == TM_PREC_FP64) {
    const double target = opts->rtol * opts->rtol * ff;
    int left = opts->max_iter;
    double rel = 0;
    TM_CUDA(ctx, cudaMemsetAsync(w.q, 0, n * sizeof(double), st));
    for (int restart = 0; restart < 8; ++restart) {
      // r = f - A u (true residual), p = Dinv r
      rc = timed_apply<double>(ctx, w.ce64, u_dev, w.q, w.part64, nullptr, nullptr, true, nullptr);
      if (rc) return rc;
      out.fp64_applies++;
      rc = init_run(ctx, 0.0, target, left);
      if (rc) return rc;
      TM_CUDA(ctx, launch_start<double>(f_dev, w.q, 1.0, w.r, w.p, w.dinv, n, solve_scalars(ctx), w.red, w.ticket + 2, st));
      ctx->launches += 1;
      int it = 0, nf = 0;
      rc = run_cg<double, double>(ctx, check, graphs, &it, &nf, w.ce64, w.part64, u_dev, w.r, w.p, w.q, w.dinv);
      if (rc) return rc;
      out.iterations += it;
      out.fp64_applies += it;
      left -= it;
      if (nf) return fail(ctx, TM_ENONFINITE, "non-finite value in CG");
      // verify with the true residual
      rc = timed_apply<double>(ctx, w.ce64, u_dev, w.q, w.part64, nullptr, nullptr, true, nullptr);
      if (rc) return rc;
      out.fp64_applies++;
      TM_CUDA(ctx, launch_residual64(f_dev, w.q, nullptr, n, rr_dev, w.red, w.ticket + 1, st));
      ctx->launches += 1;
      double rr = 0;
      rc = read_scalar(ctx, rr_dev, &rr);
      if (rc) return rc;
      rel = std::sqrt(rr / ff);
      if (rel <= opts->rtol || left <= 0) break;
    }
    out.sweeps = 1;
    out.rel_residual = rel;
    if (rel > opts->rtol) status = TM_ENOTCONVERGED;
  } else {
    // FP32-operator CG with reliable updates: the FP32 run continues until its residual
    // has dropped by inner_rtol from the largest value since the last update; then the
    // FP32 correction is added to u in FP64, the residual is replaced by the FP64 true
    // residual f - A u (rescaled to unit norm), and CG continues with the kept search
    // direction, made orthogonal to the new residual (no restart).
    const double delta = opts->inner_rtol > 0 ? opts->inner_rtol : 0.1;
    int left = opts->max_iter;
    double rel = 0, scale_old = 0;
    bool first = true;
    if (twolevel) {   // finished below, while the first true residual is computed
      rc = coarse_setup_begin(ctx, rho_dev, &out.setup_seconds);
      if (rc) return rc;
      out.coarse_levels = ctx->coarse.nlev;
    }
    TM_CUDA(ctx, cudaMemsetAsync(w.q32, 0, n * sizeof(float), st));
    TM_CUDA(ctx, cudaMemsetAsync(w.x32, 0, n * sizeof(float), st));
    for (int sweep = 0; sweep < 4096; ++sweep) {
      rc = timed_apply<double>(ctx, w.ce64, u_dev, w.q, w.part64, nullptr, nullptr, true, nullptr);
      if (rc) return rc;
      out.fp64_applies++;
      TM_CUDA(ctx, launch_residual64(f_dev, w.q, w.r, n, rr_dev, w.red, w.ticket + 1, st));
      ctx->launches += 1;
      if (twolevel && sweep == 0) {
        rc = coarse_setup_end(ctx, &out.setup_seconds);
        if (rc) return rc;
      }
      double rr = 0;
      rc = read_scalar(ctx, rr_dev, &rr);
      if (rc) return rc;
      if (!std::isfinite(rr)) return fail(ctx, TM_ENONFINITE, "non-finite residual");
      rel = std::sqrt(rr / ff);
      if (rel <= opts->rtol || left <= 0) break;
      out.sweeps++;
      const double scale = 1.0 / std::sqrt(rr);
      // stop a little past the outer target
      const double abs_stop = 0.25 * opts->rtol * opts->rtol * ff / rr;
      if (first) {
        rc = init_run(ctx, delta * delta, abs_stop, left);
        if (rc) return rc;
        TM_CUDA(ctx, launch_start<float>(w.r, nullptr, scale, w.r32, w.p32, w.dinv32, n, solve_scalars(ctx), w.red,
                                         w.ticket + 2, st));
        if (twolevel) {
          rc = enqueue_twolevel(ctx, 1, w.r32, w.p32, w.dinv32, nu);
          if (rc) return rc;
        }
        first = false;
      } else {
        TM_CUDA(ctx, launch_replace(w.r, scale, scale / scale_old, w.r32, w.p32, w.dinv32, n, abs_stop, left,
                                    solve_scalars(ctx), w.red, w.ticket + 2, st, twolevel));
        ctx->launches += twolevel ? 0 : 1;
        if (twolevel) {
          rc = enqueue_twolevel(ctx, 2, w.r32, w.p32, w.dinv32, nu);
          if (rc) return rc;
        }
      }
      ctx->launches += 1;
      scale_old = scale;
      int it = 0, nf = 0;
      rc = run_cg<float, float>(ctx, check, graphs, &it, &nf, w.ce32, w.part32, w.x32, w.r32, w.p32, w.q32,
                                w.dinv32, twolevel ? TM_PRECOND_TWOLEVEL : TM_PRECOND_JACOBI, nu);
      if (rc) return rc;
      out.iterations += it;
      out.fp32_applies += it;
      left -= it;
      if (nf) return fail(ctx, TM_ENONFINITE, "non-finite value in the FP32 iteration");
      TM_CUDA(ctx, launch_correct(u_dev, w.x32, 1.0 / scale, n, st));
      ctx->launches += 1;
    }
    out.rel_residual = rel;
    if (rel > opts->rtol) status = TM_ENOTCONVERGED;
  }
  TM_CUDA(ctx, cudaEventRecord(ctx->ev1, st));
  TM_CUDA(ctx, cudaEventSynchronize(ctx->ev1));
  float ms = 0;
  TM_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  out.seconds = ms * 1e-3;
  rc = drain_profile(ctx, false);
  if (rc) return rc;
  if (stats) *stats = out;
  if (status == TM_ENOTCONVERGED) return fail(ctx, status, "max_iter reached before rtol");
  return status;
} catch (...) {
  return exception_status(ctx);
}

int tm_pcg_solve_multi(tm_ctx *ctx, int nrhs, const double *rho_dev, const double *f_dev, double *u_dev,
                       const tm_solve_opts *opts, tm_solve_stats *stats) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !f_dev || !u_dev || !opts) return fail(ctx, TM_EINVAL, "null pointer");
  if (nrhs < 1 || nrhs > kMaxRhs) return fail(ctx, TM_EINVAL, "nrhs must be in [1, " + std::to_string(kMaxRhs) + "]");
  if (opts->precision != TM_PREC_MIXED) return fail(ctx, TM_EINVAL, "multi-load solves are TM_PREC_MIXED only");
  if (opts->precond != TM_PRECOND_JACOBI && opts->precond != TM_PRECOND_TWOLEVEL)
    return fail(ctx, TM_EINVAL, "unknown preconditioner");
  if (!(opts->rtol > 0) || opts->max_iter < 1) return fail(ctx, TM_EINVAL, "need rtol > 0 and max_iter >= 1");
  const bool twolevel = opts->precond == TM_PRECOND_TWOLEVEL;
  const int nu = opts->smooth_sweeps > 0 ? opts->smooth_sweeps : 1;
  const bool graphs = opts->no_graphs == 0;
  const DeviceMesh &m = ctx->dm;
  Work &w = ctx->w;
  cudaStream_t st = ctx->stream;
  const int64_t n = 3 * m.Nn;
  const int check = opts->check_every > 0 ? opts->check_every : 32;
  const double delta = opts->inner_rtol > 0 ? opts->inner_rtol : 0.1;
  const int pstride = 16 * device_sms();   // reduction partials per load case
  if (!w.mvec) {
    TM_CUDA(ctx, alloc(w.owned, w.bytes, &w.mvec, (size_t)kMaxRhs * 4 * n));
    TM_CUDA(ctx, alloc(w.owned, w.bytes, &w.mr64, (size_t)kMaxRhs * n));
    TM_CUDA(ctx, alloc(w.owned, w.bytes, &w.msc, (size_t)kMaxRhs));
    TM_CUDA(ctx, alloc(w.owned, w.bytes, &w.mdotp, (size_t)kMaxRhs * std::max(apply_ctas(m), 1)));
    TM_CUDA(ctx, alloc(w.owned, w.bytes, &w.mred, (size_t)kMaxRhs * pstride));
    TM_CUDA(ctx, alloc(w.owned, w.bytes, &w.mticket, (size_t)4 * kMaxRhs));
  }
  if (!w.part_multi) TM_CUDA(ctx, alloc(w.owned, w.bytes, &w.part_multi, (size_t)kMaxRhs * 3 * m.nslot));
  // kind-major: the p (q) vectors of the load cases are consecutive, as the operator reads them
  auto vec = [&](int r, int k) { return w.mvec + ((size_t)k * kMaxRhs + r) * n; };   // k: 0 x, 1 r, 2 p, 3 q
  auto scal = [&](int r) { return w.msc + r; };
  unsigned int *t_apply = w.mticket, *t_update = w.mticket + kMaxRhs, *t_finish = w.mticket + 2 * kMaxRhs;
  std::vector<tm_solve_stats> out(nrhs);
  std::memset(out.data(), 0, nrhs * sizeof(tm_solve_stats));
  TM_CUDA(ctx, cudaEventRecord(ctx->ev0, st));
  TM_CUDA(ctx, launch_coeff(m, w, rho_dev, st));
  TM_CUDA(ctx, launch_diag(m, w.ce64, nullptr, w.dinv, w.dinv32, st));
  ctx->launches += 2;
  double setup_s = 0;
  int rc;
  if (twolevel) {
    rc = coarse_setup(ctx, rho_dev, &setup_s);
    if (rc) return rc;
  }
  double *rr_dev = scal_at(ctx, 81), *ff_dev = scal_at(ctx, 82);
  std::vector<double> ff(nrhs), scale_old(nrhs, 0.0), rel(nrhs, 0.0);
  std::vector<int> left(nrhs, opts->max_iter), active(nrhs, 1), first(nrhs, 1);
  // FP64 true residual of load case r into mr64[r]; returns ||r||^2 in *rr
  auto residual = [&](int r, double *rr) -> int {
    int rc2 = timed_apply<double>(ctx, w.ce64, u_dev + (size_t)r * n, w.q, w.part64, nullptr, nullptr, true, nullptr);
    if (rc2) return rc2;
    out[r].fp64_applies++;
    TM_CUDA(ctx, launch_residual64(f_dev + (size_t)r * n, w.q, w.mr64 + (size_t)r * n, n, rr_dev, w.red,
                                   w.ticket + 1, st));
    ctx->launches += 1;
    return read_scalar(ctx, rr_dev, rr);
  };
  // start or continue load case r's CG run from its FP64 residual (reliable update)
  auto segment = [&](int r, double rr) -> int {
    const double scale = 1.0 / std::sqrt(rr);
    const double abs_stop = 0.25 * opts->rtol * opts->rtol * ff[r] / rr;
    out[r].sweeps++;
    if (first[r]) {
      SolveScalars sc0;
      std::memset(&sc0, 0, sizeof(sc0));
      sc0.stop_ratio2 = delta * delta;
      sc0.stop_abs_rr = abs_stop;
      sc0.max_it = left[r];
      TM_CUDA(ctx, cudaMemcpyAsync(scal(r), &sc0, sizeof(sc0), cudaMemcpyHostToDevice, st));
      TM_CUDA(ctx, cudaMemsetAsync(vec(r, 0), 0, n * sizeof(float), st));
      TM_CUDA(ctx, launch_start<float>(w.mr64 + (size_t)r * n, nullptr, scale, vec(r, 1), vec(r, 2), w.dinv32, n,
                                       scal(r), w.red, w.ticket + 2, st));
      TM_CUDA(ctx, cudaStreamSynchronize(st));   // sc0 lives on the host stack
      if (twolevel) {
        rc = enqueue_twolevel_cases(ctx, 1, vec(0, 1), vec(0, 2), n, w.dinv32, nu, w.msc, r, 1, w.mred, pstride,
                                    t_finish);
        if (rc) return rc;
      }
      first[r] = 0;
    } else {
      TM_CUDA(ctx, launch_replace(w.mr64 + (size_t)r * n, scale, scale / scale_old[r], vec(r, 1), vec(r, 2), w.dinv32,
                                  n, abs_stop, left[r], scal(r), w.red, w.ticket + 2, st, twolevel));
      ctx->launches += twolevel ? 0 : 1;
      if (twolevel) {
        rc = enqueue_twolevel_cases(ctx, 2, vec(0, 1), vec(0, 2), n, w.dinv32, nu, w.msc, r, 1, w.mred, pstride,
                                    t_finish);
        if (rc) return rc;
      }
    }
    ctx->launches += 1;
    scale_old[r] = scale;
    return TM_OK;
  };
  for (int r = 0; r < nrhs; ++r) {
    TM_CUDA(ctx, launch_residual64(f_dev + (size_t)r * n, nullptr, nullptr, n, ff_dev, w.red, w.ticket + 1, st));
    ctx->launches += 1;
    rc = read_scalar(ctx, ff_dev, &ff[r]);
    if (rc) return rc;
    if (!std::isfinite(ff[r])) return fail(ctx, TM_ENONFINITE, "non-finite load vector");
    if (ff[r] == 0.0) {
      TM_CUDA(ctx, cudaMemsetAsync(u_dev + (size_t)r * n, 0, n * sizeof(double), st));
      active[r] = 0;
      continue;
    }
    double rr = 0;
    rc = residual(r, &rr);
    if (rc) return rc;
    if (!std::isfinite(rr)) return fail(ctx, TM_ENONFINITE, "non-finite residual");
    rel[r] = std::sqrt(rr / ff[r]);
    if (rel[r] <= opts->rtol) {
      active[r] = 0;
      continue;
    }
    rc = segment(r, rr);
    if (rc) return rc;
  }
  // inactive load cases are marked done so that the kernels skip them
  for (int r = 0; r < nrhs; ++r)
    if (!active[r]) {
      const int one = 1;
      TM_CUDA(ctx, cudaMemcpyAsync(&scal(r)->done, &one, sizeof(int), cudaMemcpyHostToDevice, st));
      TM_CUDA(ctx, cudaStreamSynchronize(st));
    }
  // one lockstep iteration for all cases: the multi-vector operator pass, the update of every case
  // in one launch, then (two-level) the coarse step of every case in one launch sequence or
  // (Jacobi) each case's p update; cases whose run is done return at once
  auto iteration = [&]() -> int {
    TM_CUDA(ctx, launch_apply_multi(m, nrhs, w.ce32, vec(0, 2), vec(0, 3), w.part_multi, w.mdotp, scal(0), t_apply,
                                    ctx->stream));
    TM_CUDA(ctx, launch_update_nodes_cases(nrhs, vec(0, 0), vec(0, 2), vec(0, 3), vec(0, 1), n, w.dinv32, m.Nn,
                                           m.sh_of_node, m.sh_ptr, w.part_multi, 3 * m.nslot, w.msc, w.mred,
                                           t_update, ctx->stream, twolevel));
    ctx->launches += 2;
    if (twolevel)
      return enqueue_twolevel_cases(ctx, 0, vec(0, 1), vec(0, 2), n, w.dinv32, nu, w.msc, 0, nrhs, w.mred, pstride,
                                    t_finish);
    for (int r = 0; r < nrhs; ++r) {
      TM_CUDA(ctx, launch_pupdate<float>(vec(r, 2), vec(r, 1), w.dinv32, n, scal(r), ctx->stream));
      ctx->launches += 1;
    }
    return TM_OK;
  };
  cudaGraphExec_t exec = nullptr;
  int graph_launches = 0;
  if (graphs) {
    // a batch of `check` lockstep iterations captured once on the library stream and replayed
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->gstream;
    const int64_t l0 = ctx->launches;
    cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
    rc = TM_OK;
    for (int k = 0; k < check && e == cudaSuccess && rc == TM_OK; ++k) rc = iteration();
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(ctx->gstream, &graph);
    ctx->stream = user;
    graph_launches = (int)(ctx->launches - l0);
    ctx->launches = l0;
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(ctx, TM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    if (rc) {
      cudaGraphDestroy(graph);
      return rc;
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, TM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  struct GraphGuard {
    cudaGraphExec_t g;
    ~GraphGuard() { if (g) cudaGraphExecDestroy(g); }
  } guard{exec};
  std::vector<SolveScalars> hs(nrhs);
  auto any_active = [&] {
    for (int r = 0; r < nrhs; ++r)
      if (active[r]) return true;
    return false;
  };
  while (any_active()) {
    if (exec) {
      TM_CUDA(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
      TM_CUDA(ctx, cudaStreamWaitEvent(ctx->gstream, ctx->ev_fork, 0));
      TM_CUDA(ctx, cudaGraphLaunch(exec, ctx->gstream));
      TM_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->gstream));
      TM_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
      ctx->launches += graph_launches;
    } else {
      for (int k = 0; k < check; ++k) {
        rc = iteration();
        if (rc) return rc;
      }
    }
    for (int r = 0; r < nrhs; ++r)
      TM_CUDA(ctx, cudaMemcpyAsync(&hs[r], scal(r), sizeof(SolveScalars), cudaMemcpyDeviceToHost, st));
    TM_CUDA(ctx, cudaStreamSynchronize(st));
    for (int r = 0; r < nrhs; ++r) {
      if (!active[r] || !hs[r].done) continue;
      // the run of load case r reached its replacement point (or its limit)
      out[r].iterations += hs[r].it;
      out[r].fp32_applies += hs[r].it;
      left[r] -= hs[r].it;
      if (hs[r].nonfinite) return fail(ctx, TM_ENONFINITE, "non-finite value in the FP32 iteration");
      TM_CUDA(ctx, launch_correct(u_dev + (size_t)r * n, vec(r, 0), 1.0 / scale_old[r], n, st));
      ctx->launches += 1;
      double rr = 0;
      rc = residual(r, &rr);
      if (rc) return rc;
      if (!std::isfinite(rr)) return fail(ctx, TM_ENONFINITE, "non-finite residual");
      rel[r] = std::sqrt(rr / ff[r]);
      if (rel[r] <= opts->rtol || left[r] <= 0) {
        active[r] = 0;       // its scalars keep done set: the kernels skip it
        continue;
      }
      rc = segment(r, rr);
      if (rc) return rc;
    }
  }
  TM_CUDA(ctx, cudaEventRecord(ctx->ev1, st));
  TM_CUDA(ctx, cudaEventSynchronize(ctx->ev1));
  float ms = 0;
  TM_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  rc = drain_profile(ctx, false);
  if (rc) return rc;
  int status = TM_OK;
  for (int r = 0; r < nrhs; ++r) {
    out[r].rel_residual = rel[r];
    out[r].seconds = ms * 1e-3;
    out[r].setup_seconds = setup_s;
    out[r].coarse_levels = twolevel ? ctx->coarse.nlev : 0;
    if (rel[r] > opts->rtol) status = TM_ENOTCONVERGED;
  }
  if (stats) std::memcpy(stats, out.data(), nrhs * sizeof(tm_solve_stats));
  if (status == TM_ENOTCONVERGED) return fail(ctx, status, "max_iter reached before rtol");
  return status;
} catch (...) {
  return exception_status(ctx);
}

int tm_sensitivity(tm_ctx *ctx, const double *rho_dev, const double *u_full_dev, double *dc_dev,
                   double *compliance_out) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !u_full_dev || !dc_dev) return fail(ctx, TM_EINVAL, "null pointer");
  double *cdev = scal_at(ctx, 80);
  TM_CUDA(ctx, launch_sensitivity(ctx->dm, rho_dev, u_full_dev, dc_dev, ctx->w.red, ctx->w.ticket + 3, cdev,
                                  ctx->stream));
  ctx->launches += 1;
  if (compliance_out) return read_scalar(ctx, cdev, compliance_out);
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_filter(tm_ctx *ctx, const double *rho_dev, const double *x_dev, double rmin, int mode, double *out_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !x_dev || !out_dev) return fail(ctx, TM_EINVAL, "null pointer");
  if (mode != 0 && mode != 1) return fail(ctx, TM_EINVAL, "mode must be 0 or 1");
  if (!(rmin > 0) || rmin > 4.0 * ctx->dm.hmin) return fail(ctx, TM_EINVAL, "rmin must be in (0, 4 h_min]");
  TM_CUDA(ctx, launch_filter(ctx->dm, rho_dev, x_dev, rmin, mode, out_dev, ctx->stream));
  ctx->launches += 1;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_oc_update(tm_ctx *ctx, const double *rho_dev, const double *dc_dev, double volfrac, double move, double eta,
                 double rho_min, double *rho_new_dev, double *change_out) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev || !dc_dev || !rho_new_dev) return fail(ctx, TM_EINVAL, "null pointer");
  if (!(volfrac > 0 && volfrac <= 1) || !(move > 0) || !(eta > 0) || !(rho_min > 0 && rho_min < 1))
    return fail(ctx, TM_EINVAL, "bad OC parameters");
  OcState s;
  std::memset(&s, 0, sizeof(s));
  s.target = volfrac * ctx->dm.volume;
  s.tol = 1e-12;
  TM_CUDA(ctx, cudaMemcpyAsync(oc_state(ctx), &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream));
  if (!ctx->w.octab) TM_CUDA(ctx, alloc(ctx->w.owned, ctx->w.bytes, &ctx->w.octab, (size_t)ctx->dm.Ne));
  const DeviceMesh &m = ctx->dm;
  double *part = ctx->w.red;
  unsigned int *tk = ctx->w.ticket + 4;
  TM_CUDA(ctx, launch_oc_init(m, rho_dev, dc_dev, eta, move, rho_min, ctx->w.octab, part, tk, oc_state(ctx),
                              ctx->stream));
  // the search usually ends within 10 launches; the state is read back between rounds of launches
  // so that few launches run after it has ended (at most 64 in all)
  int launched = 0;
  for (int round = 0; round < 8; ++round) {
    const int n = round == 0 ? 10 : 6;
    TM_CUDA(ctx, launch_oc_search(m, eta, ctx->w.octab, part, tk, oc_state(ctx), n, ctx->stream));
    launched += n;
    TM_CUDA(ctx, cudaMemcpyAsync(&s, oc_state(ctx), sizeof(s), cudaMemcpyDeviceToHost, ctx->stream));
    TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (s.done || launched >= 64) break;
  }
  TM_CUDA(ctx, launch_oc_final(m, rho_dev, eta, ctx->w.octab, rho_new_dev, part, tk, oc_state(ctx), ctx->stream));
  ctx->launches += launched + 2;
  if (change_out) return read_scalar(ctx, &oc_state(ctx)->change, change_out);
  TM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

// ---------------------------------------------------------------- two-level preconditioner
int tm_coarse_setup(tm_ctx *ctx, const double *rho_dev, int32_t *levels_out, int32_t *shapes_out) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  if (!rho_dev) return fail(ctx, TM_EINVAL, "null pointer");
  int rc = coarse_setup(ctx, rho_dev, nullptr);
  if (rc) return rc;
  const CoarseHierarchy &h = ctx->coarse;
  if (levels_out) *levels_out = h.nlev;
  if (shapes_out)
    for (int l = 0; l < h.nlev; ++l) {
      shapes_out[3 * l] = h.lev[l].X;
      shapes_out[3 * l + 1] = h.lev[l].Y;
      shapes_out[3 * l + 2] = h.lev[l].Z;
    }
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

#define TM_CHECK_COARSE(ctx)                                                                 \
  do {                                                                                       \
    if (!(ctx)->coarse_ready) return fail(ctx, TM_ESTATE, "no two-level set-up for this mesh"); \
  } while (0)

int tm_coarse_cells(tm_ctx *ctx, int level, float *K_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  TM_CHECK_COARSE(ctx);
  const CoarseHierarchy &h = ctx->coarse;
  if (level < 0 || level >= h.nlev || !K_dev) return fail(ctx, TM_EINVAL, "bad level or null pointer");
  const CoarseLevel &c = h.lev[level];
  TM_CUDA(ctx, cudaMemcpyAsync(K_dev, c.K, 576 * (size_t)c.X * c.Y * c.Z * sizeof(float), cudaMemcpyDeviceToDevice,
                               ctx->stream));
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_coarse_apply(tm_ctx *ctx, int level, const float *x_dev, float *y_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  TM_CHECK_COARSE(ctx);
  const CoarseHierarchy &h = ctx->coarse;
  if (level < 0 || level >= h.nlev || !x_dev || !y_dev) return fail(ctx, TM_EINVAL, "bad level or null pointer");
  TM_CUDA(ctx, coarse_level_apply_launch(h, level, x_dev, y_dev, ctx->stream));
  ctx->launches += 1;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_coarse_restrict(tm_ctx *ctx, const float *r_dev, float *b0_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  TM_CHECK_COARSE(ctx);
  if (!r_dev || !b0_dev) return fail(ctx, TM_EINVAL, "null pointer");
  const CoarseHierarchy &h = ctx->coarse;
  TM_CUDA(ctx, coarse_restrict_launch(ctx->dm, h, r_dev, 3 * ctx->dm.Nn, false, nullptr, 0, 1, ctx->stream));
  TM_CUDA(ctx, cudaMemcpyAsync(b0_dev, h.lev[0].b, 3 * (size_t)h.lev[0].nodes * sizeof(float),
                               cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->launches += 2;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_coarse_prolong(tm_ctx *ctx, const float *v0_dev, float *y_dev) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  TM_CHECK_COARSE(ctx);
  if (!v0_dev || !y_dev) return fail(ctx, TM_EINVAL, "null pointer");
  TM_CUDA(ctx, coarse_prolong_launch(ctx->dm, ctx->coarse, v0_dev, y_dev, ctx->stream));
  ctx->launches += 1;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

int tm_coarse_vcycle(tm_ctx *ctx, const float *b0_dev, float *x0_dev, int nu) try {
  TM_CHECK_CTX(ctx);
  TM_CHECK_MESH(ctx);
  TM_CHECK_COARSE(ctx);
  if (!b0_dev || !x0_dev || nu < 1) return fail(ctx, TM_EINVAL, "null pointer or nu < 1");
  const CoarseHierarchy &h = ctx->coarse;
  const size_t bytes = 3 * (size_t)h.lev[0].nodes * sizeof(float);
  TM_CUDA(ctx, cudaMemcpyAsync(h.lev[0].b, b0_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  TM_CUDA(ctx, coarse_first_sweep_launch(h, ctx->stream));
  int nl = 0;
  TM_CUDA(ctx, coarse_vcycle_launch(h, nu, nullptr, 0, 1, ctx->stream, &nl));
  TM_CUDA(ctx, cudaMemcpyAsync(x0_dev, h.lev[0].x, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->launches += 1 + nl;
  return TM_OK;
} catch (...) {
  return exception_status(ctx);
}

}  // extern "C"

