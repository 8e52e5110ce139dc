// Operator kernels: y = C^T K(rho) C x on the A-space (paper Eq. 6-7), the
// element coefficients c_e = (Emin + rho_e^p (E0 - Emin)) h_e (Eq. 2), the
// Jacobi diagonal of Sec. 5 and the expansion u_full = C u (Eq. 9).
//
// Operator layout (tables built by mesh_host.cpp).  Elements are grouped in
// blocks of 256 consecutive elements; a block's local nodes are its regular
// nodes followed by the hanging nodes its elements use; each block has one
// 16-byte-aligned record: corner -> local id per element, local -> global node,
// shared-node partial positions, hanging masters, and per-local-node inverse
// lists (the (element, corner) slots it collects, plus fold entries naming the
// hanging nodes it is a master of).
//
// One CTA per block.  The block's record is staged into shared memory with
// cp.async, then the node values it names (zero-filled for Dirichlet nodes):
//   1. hanging nodes take the (bi)linear interpolation of their masters (C);
//   2. one thread per element gathers its 8 corners and computes c_e K0 X_e in
//      the symmetry-adapted basis (element.cuh) into a per-element slot buffer;
//   3. hanging nodes sum their slots; regular nodes sum their slots plus
//      w * (sum) of every hanging node they are a master of (C^T) -- a fixed
//      summation order, no atomics, bitwise reproducible;
//   4. nodes touched only by this block are stored to y; nodes shared with
//      other blocks are stored to their partial slots (node-major), which the CG
//      update or a second kernel sums in ascending block order.  Hanging DOFs of
//      y are set to 0.
// The element energies c_e X_e^T K0 X_e can be accumulated on the fly: their
// sum is CG's p^T A p.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "brick.cuh"
#include "element.cuh"
#include "pcg.cuh"
#include "pdl.cuh"
#include "reduce.cuh"
#include "tm_internal.h"

namespace amr {

constexpr int kApplyThreads = kBlockElems;  // one thread per element of a block
constexpr int kRow = kSlotRow;              // padded per-element row of the slot buffer

template <typename T>
struct ApplyParams {
  const uint4 *brec;        // per-block records
  const int32_t *rec_off;   // record ranges in 16-byte units
  const int32_t *rec_skip;  // per block: 16-byte units of lcorner and elist, read from global memory
  const T *ce;
  const T *x;
  T *y;
  T *part;
  double *dotp;     // per-CTA partials of x^T A x (nullptr: skip)
  SolveScalars *sc; // with dotp: the last CTA sets sc->pq and sc->alpha = sc->rz / pq
  unsigned int *ticket;
  const int *done;  // skip the launch when set (nullptr: never)
  ModalBlocks<T> K;
  int nblk;
  int max_local;    // local nodes of the largest block
  int rec_bytes;    // record buffer size (largest record, multiple of 16)
  int ahead;        // CTAs resident on the GPU: block b prefetches the record of b + ahead into L2
  BrickTables bricks;  // CTAs nblk .. take 4 bricks each (brick.cuh)
};


// Shared memory: XY (per-element slots) | R (3 values per local node) | record.
template <typename T>
__host__ __device__ __forceinline__ size_t val_buf_bytes(int max_local) {
  return ((sizeof(T) * 3 * (size_t)max_local) + 15) / 16 * 16;
}
template <typename T>
__host__ __device__ __forceinline__ size_t xy_bytes() {
  return ((sizeof(T) * (size_t)kApplyThreads * kRow) + 15) / 16 * 16;
}
template <typename T>
size_t apply_smem_bytes(int max_local, int rec_bytes) {
  return std::max(xy_bytes<T>() + val_buf_bytes<T>(max_local) + (size_t)rec_bytes, brick_smem_bytes<T>());
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// copies `bytes` (4 or 8) and zero-fills the destination when `fill_zero`
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *dst, const void *src, bool fill_zero) {
  const int srcsz = fill_zero ? 0 : BYTES;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
               "r"(srcsz)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Record of block `blk` into `rec` (all threads; an empty group past the end): its 64-byte header
// and its sections from lnode on (lcorner and elist, read once per element, stay in global
// memory), so that the sections after the header sit 16 * skip bytes below their record offsets.
__device__ __forceinline__ void issue_record(const uint4 *brec, const int32_t *rec_off, const int32_t *rec_skip,
                                             int blk, int nblk, uint4 *rec) {
  if (blk < nblk) {
    const int r0 = rec_off[blk], nr = rec_off[blk + 1] - r0, skip = rec_skip[blk];
    for (int i = threadIdx.x; i < nr - skip; i += kApplyThreads)
      cp_async16(rec + i, brec + r0 + (i < 4 ? i : i + skip));
  }
  cp_async_commit();
}

// Node values of the block whose record is in `rec` into `R`: consecutive threads copy
// consecutive words (word w is component w % 3 of local node w / 3), so a run of consecutive node
// ids is read with contiguous, coalesced requests.
template <typename T>
__device__ __forceinline__ void issue_values(const uint4 *rec, int skip_bytes, const T *x, T *R, bool valid) {
  if (valid) {
    const int *hdr = reinterpret_cast<const int *>(rec);
    const int nreg = hdr[2];
    const uint32_t *lnode =
        reinterpret_cast<const uint32_t *>(reinterpret_cast<const unsigned char *>(rec) + hdr[11] - skip_bytes);
    for (int wd = threadIdx.x; wd < 3 * nreg; wd += kApplyThreads) {
      const int i = wd / 3, c = wd - 3 * i;
      const uint32_t gw = lnode[i];
      cp_async_small<sizeof(T)>(R + wd, x + 3 * (size_t)(gw & 0x7FFFFFFFu) + c, (gw >> 31) != 0);
    }
  }
  cp_async_commit();
}

template <typename T>
__global__ void __launch_bounds__(kApplyThreads, (sizeof(T) == 4 ? 4 : 2) * 256 / kApplyThreads)
    apply_blocks_kernel(ApplyParams<T> P) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (P.done && *(volatile const int *)P.done) return;
  double dot = 0.0;
  if (blockIdx.x >= P.nblk) {
    const int brick = (blockIdx.x - P.nblk) * kBricksPerCta + threadIdx.x / kBrickElems;
    if (P.dotp) dot = brick_pass<T, true>(P.bricks, brick, P.ce, P.x, P.y, P.part, P.K, smem_raw);
    else brick_pass<T, false>(P.bricks, brick, P.ce, P.x, P.y, P.part, P.K, smem_raw);
  } else {
  T *XY = reinterpret_cast<T *>(smem_raw);
  T *R = reinterpret_cast<T *>(smem_raw + xy_bytes<T>());
  uint4 *rec = reinterpret_cast<uint4 *>(smem_raw + xy_bytes<T>() + val_buf_bytes<T>(P.max_local));
  const int tid = threadIdx.x;
  const int b = blockIdx.x;
  // record, then the node values it names: every copy of a stage in flight at once
  issue_record(P.brec, P.rec_off, P.rec_skip, b, P.nblk, rec);
  const int skip_bytes = 16 * P.rec_skip[b];
  const unsigned char *gb = reinterpret_cast<const unsigned char *>(P.brec + P.rec_off[b]);   // the record in global memory
  // the record of the block that starts about one resident wave later, into L2 (one bulk
  // prefetch; records are 16-byte aligned multiples of 16 bytes)
  if (tid == 0 && P.ahead > 0 && b + P.ahead < P.nblk) {
    const int r0 = P.rec_off[b + P.ahead], nr = P.rec_off[b + P.ahead + 1] - r0;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(P.brec + r0), "r"(16 * nr) : "memory");
  }
  cp_async_wait<0>();
  __syncthreads();
  // the element's corner codes and coefficient (global memory), in flight with the values
  uint4 cw = make_uint4(0, 0, 0, 0);
  T coef = T(0);
  {
    const int *h0 = reinterpret_cast<const int *>(rec);
    if (tid < h0[1]) {
      cw = reinterpret_cast<const uint4 *>(gb + h0[10])[tid];
      coef = P.ce[reinterpret_cast<const int *>(gb + h0[12])[tid]];
    }
  }
  issue_values<T>(rec, skip_bytes, P.x, R, true);
  cp_async_wait<0>();
  __syncthreads();

  const int *hdr = reinterpret_cast<const int *>(rec);
  const unsigned char *rb = reinterpret_cast<const unsigned char *>(rec);
  const int ne = hdr[1], nreg = hdr[2], nshared = hdr[3], nhang = hdr[4];
  const int *lslot = reinterpret_cast<const int *>(rb + hdr[6] - skip_bytes);
  const uint2 *hent = reinterpret_cast<const uint2 *>(rb + hdr[7] - skip_bytes);
  const uint16_t *ip = reinterpret_cast<const uint16_t *>(rb + hdr[8] - skip_bytes);
  const uint16_t *iv = reinterpret_cast<const uint16_t *>(rb + hdr[9] - skip_bytes);
  const uint32_t *lnode = reinterpret_cast<const uint32_t *>(rb + hdr[11] - skip_bytes);

  // 1. hanging nodes: (bi)linear interpolation of their masters (C)
  for (int j = tid; j < nhang; j += kApplyThreads) {
    const uint2 mw = hent[j];
    const int m0 = mw.x & 0xFFFF, m1 = mw.x >> 16, m2 = mw.y & 0xFFFF, m3 = mw.y >> 16;
    T *d = R + 3 * (nreg + j);
    if (m2 == 0xFFFF) {
#pragma unroll
      for (int c = 0; c < 3; ++c) d[c] = T(0.5) * (R[3 * m0 + c] + R[3 * m1 + c]);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        d[c] = T(0.25) * ((R[3 * m0 + c] + R[3 * m1 + c]) + (R[3 * m2 + c] + R[3 * m3 + c]));
    }
  }
  __syncthreads();
  // 2. element operator: gather the 8 corners, results into the slots; x^T A x is
  // the sum of the element energies c_e X_e^T K0 X_e (C and the Dirichlet zeros are
  // already in X_e)
  if (tid < ne) {
    const int code[8] = {(int)(cw.x & 0xFFFF), (int)(cw.x >> 16), (int)(cw.y & 0xFFFF), (int)(cw.y >> 16),
                         (int)(cw.z & 0xFFFF), (int)(cw.z >> 16), (int)(cw.w & 0xFFFF), (int)(cw.w >> 16)};
    T X[24], Y[24];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      X[3 * k] = R[3 * code[k]];
      X[3 * k + 1] = R[3 * code[k] + 1];
      X[3 * k + 2] = R[3 * code[k] + 2];
    }
    if (P.dotp) dot = (double)element_op<T, kOpBoth>(X, Y, coef, P.K);
    else element_op<T, kOpApply>(X, Y, coef, P.K);
#pragma unroll
    for (int j = 0; j < 24; ++j) XY[tid * kRow + j] = Y[j];
  }
  __syncthreads();
  // 3a. hanging nodes sum their slots
  for (int j = tid; j < nhang; j += kApplyThreads) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    const int q1 = ip[nreg + j + 1];
    for (int q = ip[nreg + j]; q < q1; ++q) {
      const T *d = XY + iv[q];
      s0 += d[0]; s1 += d[1]; s2 += d[2];
    }
    T *r = R + 3 * (nreg + j);
    r[0] = s0; r[1] = s1; r[2] = s2;
  }
  __syncthreads();
  // 3b/4. regular nodes: own slots + folded hanging sums (C^T), then store
  for (int i = tid; i < nreg; i += kApplyThreads) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    const int q1 = ip[i + 1];
    for (int q = ip[i]; q < q1; ++q) {
      const int p = iv[q];
      if (!(p & kFoldBit)) {
        const T *d = XY + p;
        s0 += d[0]; s1 += d[1]; s2 += d[2];
      } else {
        const T w = (p & kQuarterBit) ? T(0.25) : T(0.5);
        const T *r = R + 3 * (nreg + (p & (kQuarterBit - 1)));
        s0 += w * r[0]; s1 += w * r[1]; s2 += w * r[2];
      }
    }
    const uint32_t gw = lnode[i];
    if (gw >> 31) s0 = s1 = s2 = T(0);
    if (i < nshared) {
      T *dst = P.part + 3 * (size_t)lslot[i];
      dst[0] = s0; dst[1] = s1; dst[2] = s2;
    } else {
      T *dst = P.y + 3 * (size_t)(gw & 0x7FFFFFFFu);
      dst[0] = s0; dst[1] = s1; dst[2] = s2;
    }
  }
  }
  if (P.dotp) {
    dot = block_sum<kApplyThreads>(dot);
    if (threadIdx.x == 0) P.dotp[blockIdx.x] = dot;
    if (P.sc && last_cta(P.ticket)) {
      const double pq = sum_partials<kApplyThreads>(P.dotp, gridDim.x);
      if (threadIdx.x == 0) {
        P.sc->pq = pq;
        P.sc->alpha = P.sc->rz / pq;
        if (!isfinite(pq) || !isfinite(P.sc->alpha) || pq <= 0.0) {
          P.sc->nonfinite = 1;
          P.sc->done = 1;
        }
      }
    }
  }
}

// Second pass: each shared node sums its contiguous run of partials (one per
// block touching it, in ascending block order); optionally hanging DOFs of y are
// zeroed.
template <typename T>
__global__ void __launch_bounds__(256) apply_shared_kernel(const int32_t *sh_node, const int32_t *sh_ptr, int64_t nsh,
                                                           const int32_t *hang_node, int64_t nh, const T *part, T *y,
                                                           const int *done) {
  pdl_begin();
  if (done && *(volatile const int *)done) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nsh) {
    const int g = sh_node[i];
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int j = sh_ptr[i]; j < sh_ptr[i + 1]; ++j) {
      const T *src = part + 3 * (size_t)j;
      s0 += src[0]; s1 += src[1]; s2 += src[2];
    }
    T *dst = y + 3 * (size_t)g;
    dst[0] = s0; dst[1] = s1; dst[2] = s2;
  } else if (i < nsh + nh) {
    T *dst = y + 3 * (size_t)hang_node[i - nsh];
    dst[0] = dst[1] = dst[2] = T(0);
  }
}

int device_sms() {
  static std::atomic<int> cached[kStaticMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return 152;
  int n = cached[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
  cached[dev].store(n, std::memory_order_relaxed);
  return n;
}

// One thread per item (the second pass is latency-bound: no grid-stride reuse).
int item_grid(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (int)(g < 1 ? 1 : g);
}

int shared_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 8 * device_sms()) g = 8 * device_sms();  // 8 CTAs per SM; grid-stride beyond
  return (int)g;
}

// The block pass's dynamic shared-memory opt-in on the current device: only ever raised
// (meshes of several contexts share the kernel; contexts may call from several threads).
template <typename T>
cudaError_t ensure_apply_smem(size_t smem) {
  static std::mutex mu;
  static size_t configured[kStaticMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (smem > configured[dev]) {
    e = cudaFuncSetAttribute(apply_blocks_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[dev] = smem;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_apply_blocks(const DeviceMesh &m, const T *ce, const T *x, T *y, T *part, double *energy_partials,
                                SolveScalars *sc, unsigned int *ticket, const int *done, cudaStream_t s) {
  const int rec_bytes = (m.max_rec_stage + 15) / 16 * 16;
  const size_t smem = apply_smem_bytes<T>(m.max_local, rec_bytes);
  cudaError_t e = ensure_apply_smem<T>(smem);
  if (e != cudaSuccess) return e;
  const int ahead = sizeof(T) == 4 ? m.resident_cta32 : m.resident_cta64;
  ApplyParams<T> P;
  P.brec = m.brec; P.rec_off = m.rec_off; P.rec_skip = m.rec_skip; P.ce = ce; P.x = x; P.y = y; P.part = part;
  P.dotp = energy_partials; P.sc = sc; P.ticket = ticket; P.done = done; P.nblk = m.nblk;
  for (int i = 0; i < 72; ++i) (&P.K.b[0][0][0])[i] = (T)m.modal[i];
  P.max_local = m.max_local; P.rec_bytes = rec_bytes; P.ahead = ahead;
  P.bricks = BrickTables{m.brick_tab, m.nbrick};
  if (apply_ctas(m) > 0) { const cudaError_t pe_ = launch_pdl(apply_blocks_kernel<T>, dim3(apply_ctas(m)), dim3(kApplyThreads), smem, s, P); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const DeviceMesh &m, const T *ce, const T *x, T *y, T *part, double *dot_partials,
                         SolveScalars *sc, unsigned int *ticket, bool zero_hanging, const int *done,
                         cudaStream_t s) {
  cudaError_t e = launch_apply_blocks<T>(m, ce, x, y, part, dot_partials, sc, ticket, done, s);
  if (e != cudaSuccess) return e;
  const int64_t items = m.nsh + (zero_hanging ? m.nh : 0);
  { const cudaError_t pe_ = launch_pdl(apply_shared_kernel<T>, dim3(item_grid(items)), dim3(256), 0, s, m.sh_node, m.sh_ptr, m.nsh, m.hang_node,
                                                          zero_hanging ? m.nh : 0, part, y, done); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}

// CTAs of the block pass resident on the whole GPU for this mesh's shared-memory size, in FP32
// and FP64 (queried once per mesh, outside any stream capture).
cudaError_t apply_residency(const DeviceMesh &m, int *resident32, int *resident64) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int rec_bytes = (m.max_rec_stage + 15) / 16 * 16;
  const size_t s32 = apply_smem_bytes<float>(m.max_local, rec_bytes), s64 = apply_smem_bytes<double>(m.max_local, rec_bytes);
  e = ensure_apply_smem<float>(s32);
  if (e == cudaSuccess) e = ensure_apply_smem<double>(s64);
  int b32 = 0, b64 = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, apply_blocks_kernel<float>, kApplyThreads, s32);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, apply_blocks_kernel<double>, kApplyThreads, s64);
  if (e != cudaSuccess) return e;
  *resident32 = b32 * sms;
  *resident64 = b64 * sms;
  return cudaSuccess;
}

template cudaError_t launch_apply_blocks<double>(const DeviceMesh &, const double *, const double *, double *,
                                                 double *, double *, SolveScalars *, unsigned int *, const int *,
                                                 cudaStream_t);
template cudaError_t launch_apply_blocks<float>(const DeviceMesh &, const float *, const float *, float *, float *,
                                                double *, SolveScalars *, unsigned int *, const int *, cudaStream_t);
template cudaError_t launch_apply<double>(const DeviceMesh &, const double *, const double *, double *, double *,
                                          double *, SolveScalars *, unsigned int *, bool, const int *, cudaStream_t);
template cudaError_t launch_apply<float>(const DeviceMesh &, const float *, const float *, float *, float *,
                                         double *, SolveScalars *, unsigned int *, bool, const int *, cudaStream_t);

// ---------------------------------------------------------------- coefficients
__device__ __forceinline__ double simp_power(double r, double p) {
  // exact repeated products for the common integer penalties, pow() otherwise
  if (p == 3.0) return r * r * r;
  if (p == 1.0) return r;
  if (p == 2.0) return r * r;
  if (p == 4.0) return (r * r) * (r * r);
  return pow(r, p);
}

__global__ void coeff_kernel(const int32_t *leaf, const double *rho, int64_t Ne, double E0, double Emin,
                             double penal, double h0, double *ce64, float *ce32) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    const double h = ldexp(h0, -leaf[4 * e + 3]);
    const double c = (Emin + simp_power(rho[e], penal) * (E0 - Emin)) * h;
    if (ce64) ce64[e] = c;
    ce32[e] = (float)c;
  }
}

cudaError_t launch_coeff(const DeviceMesh &m, const Work &w, const double *rho, cudaStream_t s) {
  coeff_kernel<<<shared_grid(m.Ne), 256, 0, s>>>(m.leaf, rho, m.Ne, m.E0, m.Emin, m.penal, m.h0, w.ce64, w.ce32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- no-allocation operator
// Scratch of tm_apply_K_f32_static: the FP32 coefficients (kStaticElems) followed by
// the shared-node partials (3 * kStaticSlots), 32 MiB in all, resident on every
// device that loads the library.  Host code cannot use the symbol as a device
// address; its address is fetched once per device with that device current.
static __device__ __align__(256) float g_static_scratch[kStaticElems + 3 * kStaticSlots];
static float *g_static_ptr[kStaticMaxDevices];
static std::mutex g_static_mu;   // first calls from several host threads look the address up once

cudaError_t static_scratch(int device, float **ce, float **part) {
  if (device < 0 || device >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[device] = static_cast<float *>(p);
  }
  *ce = g_static_ptr[device];
  *part = g_static_ptr[device] + kStaticElems;
  return cudaSuccess;
}

cudaError_t launch_coeff_f32(const DeviceMesh &m, const double *rho, float *ce32, cudaStream_t s) {
  coeff_kernel<<<shared_grid(m.Ne), 256, 0, s>>>(m.leaf, rho, m.Ne, m.E0, m.Emin, m.penal, m.h0, nullptr, ce32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Jacobi diagonal
// d_{n,c} = sum over the node's (element, triple) entries of c_e * q_c (c_e from
// the coefficient kernel); the
// coefficient triples q = v^T K0 v (v: the node's weights on the element's
// corners) depend on the mesh only and were tabulated on the host.
__global__ void diag_kernel(const int32_t *dg_ptr, const int32_t *dg_elem, const uint16_t *dg_q,
                            const double *dg_tab, const double *ce, const uint8_t *nflag, int64_t Nn, double *d,
                            double *dinv, float *dinv32) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < Nn; n += (int64_t)gridDim.x * blockDim.x) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int j = dg_ptr[n]; j < dg_ptr[n + 1]; ++j) {
      const double c = ce[dg_elem[j]];
      const double *q = dg_tab + 3 * dg_q[j];
      s0 += c * q[0]; s1 += c * q[1]; s2 += c * q[2];
    }
    const bool constrained = nflag[n] != 0;
    if (constrained) s0 = s1 = s2 = 1.0;
    if (d) { d[3 * n] = s0; d[3 * n + 1] = s1; d[3 * n + 2] = s2; }
    const double i0 = constrained ? 0.0 : 1.0 / s0, i1 = constrained ? 0.0 : 1.0 / s1,
                 i2 = constrained ? 0.0 : 1.0 / s2;
    if (dinv) { dinv[3 * n] = i0; dinv[3 * n + 1] = i1; dinv[3 * n + 2] = i2; }
    if (dinv32) { dinv32[3 * n] = (float)i0; dinv32[3 * n + 1] = (float)i1; dinv32[3 * n + 2] = (float)i2; }
  }
}

cudaError_t launch_diag(const DeviceMesh &m, const double *ce, double *d, double *dinv, float *dinv32,
                        cudaStream_t s) {
  diag_kernel<<<shared_grid(m.Nn), 256, 0, s>>>(m.dg_ptr, m.dg_elem, m.dg_q, m.dg_tab, ce, m.nflag, m.Nn, d, dinv,
                                                 dinv32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- C and C^T on nodes
__global__ void expand_kernel(const double *u, double *uf, const uint8_t *nflag, const int32_t *hang_index_unused,
                              int64_t Nn) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < Nn; n += (int64_t)gridDim.x * blockDim.x) {
    const bool keep = nflag[n] == 0;
    uf[3 * n] = keep ? u[3 * n] : 0.0;
    uf[3 * n + 1] = keep ? u[3 * n + 1] : 0.0;
    uf[3 * n + 2] = keep ? u[3 * n + 2] : 0.0;
  }
}

// hanging DOFs: (bi)linear interpolation of the masters (Eq. 9); a Dirichlet
// master contributes its prescribed 0.  Runs after expand_kernel.
__global__ void expand_hanging_kernel(const int32_t *hang_node, const int32_t *hang_master, int64_t nh,
                                      const uint8_t *nflag, const double *u, double *uf) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nh; i += (int64_t)gridDim.x * blockDim.x) {
    const int h = hang_node[i];
    const int nm = hang_master[4 * i + 2] < 0 ? 2 : 4;
    const double w = nm == 2 ? 0.5 : 0.25;
    double s0 = 0, s1 = 0, s2 = 0;
    for (int q = 0; q < nm; ++q) {
      const int mm = hang_master[4 * i + q];
      if (nflag[mm] & 1) continue;
      s0 += w * u[3 * mm]; s1 += w * u[3 * mm + 1]; s2 += w * u[3 * mm + 2];
    }
    if (nflag[h] & 1) s0 = s1 = s2 = 0.0;
    uf[3 * h] = s0; uf[3 * h + 1] = s1; uf[3 * h + 2] = s2;
  }
}

cudaError_t launch_expand(const DeviceMesh &m, const double *u, double *uf, cudaStream_t s) {
  expand_kernel<<<shared_grid(m.Nn), 256, 0, s>>>(u, uf, m.nflag, nullptr, m.Nn);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || m.nh == 0) return e;
  expand_hanging_kernel<<<shared_grid(m.nh), 256, 0, s>>>(m.hang_node, m.hang_master, m.nh, m.nflag, u, uf);
  return cudaGetLastError();
}

}  // namespace amr
