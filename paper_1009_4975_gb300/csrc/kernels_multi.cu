// The FP32 operator applied to several vectors at once (paper Eq. 6-9 for each):
// y_r = C^T K(rho) C x_r, r < nr; inside the multi-load CG it also sums each vector's
// element energies (p^T A p) and sets alpha, skipping vectors whose run is done.  Same tables, same per-vector arithmetic and
// summation order as the single-vector block pass (kernels_apply.cu), so each y_r
// equals a single application bit for bit; the block's record is staged into shared
// memory once for all vectors, and the node values of every vector in one stage.
//
// Shared memory: per-element slot buffer (reused vector after vector) | node values
// of the nr vectors | record.
#include <cuda_runtime.h>

#include <mutex>

#include "brick.cuh"
#include "element.cuh"
#include "pcg.cuh"
#include "pdl.cuh"
#include "reduce.cuh"
#include "tm_internal.h"

namespace amr {

namespace {

constexpr int kThreads = kBlockElems;  // one thread per element of a block
constexpr int kRowM = kSlotRow;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void copy16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void copy4(void *dst, const void *src, bool fill_zero) {
  const int srcsz = fill_zero ? 0 : 4;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(srcsz)
               : "memory");
}
__device__ __forceinline__ void copies_done() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__host__ __device__ __forceinline__ size_t slot_bytes() { return ((sizeof(float) * (size_t)kThreads * kRowM) + 15) / 16 * 16; }
__host__ __device__ __forceinline__ size_t values_bytes(int max_local) { return ((sizeof(float) * 3 * (size_t)max_local) + 15) / 16 * 16; }

struct MultiParams {
  const uint4 *brec;
  const int32_t *rec_off;
  const float *ce;
  const float *x;      // nr vectors, stride ld
  float *y;            // nr vectors, stride ld
  float *part;         // nr partial arrays, stride 3 * nslot
  int64_t ld, nslot;
  double *dotp;        // with sc: per-CTA element-energy partials, nr x gridDim.x
  SolveScalars *sc;    // per-vector CG scalars (nullptr: plain application); done vectors are skipped
  unsigned int *ticket;
  ModalBlocks<float> K;
  int nr, max_local;
  int nblk;             // CTAs nblk .. take 4 bricks each (brick.cuh), vector after vector
  BrickTables bricks;
};

__global__ void __launch_bounds__(kThreads, 2) apply_blocks_multi_kernel(MultiParams P) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *XY = reinterpret_cast<float *>(smem_raw);
  const size_t vb = values_bytes(P.max_local);
  unsigned char *vals = smem_raw + slot_bytes();
  uint4 *rec = reinterpret_cast<uint4 *>(vals + (size_t)P.nr * vb);
  const int tid = threadIdx.x;
  const int b = blockIdx.x;
  if (b >= P.nblk) {
    const int brick = (b - P.nblk) * kBricksPerCta + tid / kBrickElems;
    for (int r = 0; r < P.nr; ++r) {
      if (P.sc && *(volatile const int *)&P.sc[r].done) continue;   // uniform over the CTA
      const float *x = P.x + (size_t)r * P.ld;
      float *y = P.y + (size_t)r * P.ld;
      float *part = P.part + (size_t)r * 3 * P.nslot;
      if (P.sc) {
        double energy = brick_pass<float, true>(P.bricks, brick, P.ce, x, y, part, P.K, smem_raw);
        energy = block_sum<kThreads>(energy);
        if (tid == 0) P.dotp[(size_t)r * gridDim.x + b] = energy;
      } else {
        brick_pass<float, false>(P.bricks, brick, P.ce, x, y, part, P.K, smem_raw);
      }
      __syncthreads();   // the lattice buffers are reused by the next vector
    }
  } else {
  {
    const int r0 = P.rec_off[b], nrec = P.rec_off[b + 1] - r0;
    for (int i = tid; i < nrec; i += kThreads) copy16(rec + i, P.brec + r0 + i);
    copies_done();
    __syncthreads();
  }
  const int *hdr = reinterpret_cast<const int *>(rec);
  const unsigned char *rb = reinterpret_cast<const unsigned char *>(rec);
  const int ne = hdr[1], nreg = hdr[2], nshared = hdr[3], nhang = hdr[4];
  const int *lslot = reinterpret_cast<const int *>(rb + hdr[6]);
  const uint2 *hent = reinterpret_cast<const uint2 *>(rb + hdr[7]);
  const uint16_t *ip = reinterpret_cast<const uint16_t *>(rb + hdr[8]);
  const uint16_t *iv = reinterpret_cast<const uint16_t *>(rb + hdr[9]);
  const uint4 *lcorner = reinterpret_cast<const uint4 *>(rb + hdr[10]);
  const uint32_t *lnode = reinterpret_cast<const uint32_t *>(rb + hdr[11]);
  const int *elist = reinterpret_cast<const int *>(rb + hdr[12]);
  // node values of every vector (zero-filled at Dirichlet nodes), one stage
  for (int r = 0; r < P.nr; ++r) {
    float *R = reinterpret_cast<float *>(vals + (size_t)r * vb);
    const float *x = P.x + (size_t)r * P.ld;
    for (int i = tid; i < nreg; i += kThreads) {
      const uint32_t gw = lnode[i];
      const bool fixed = gw >> 31;
      const float *src = x + 3 * (size_t)(gw & 0x7FFFFFFFu);
#pragma unroll
      for (int c = 0; c < 3; ++c) copy4(R + 3 * i + c, src + c, fixed);
    }
  }
  copies_done();
  __syncthreads();
  float coef = 0.0f;
  uint4 cw = make_uint4(0, 0, 0, 0);
  if (tid < ne) {
    coef = P.ce[elist[tid]];
    cw = lcorner[tid];
  }
  const int code[8] = {(int)(cw.x & 0xFFFF), (int)(cw.x >> 16), (int)(cw.y & 0xFFFF), (int)(cw.y >> 16),
                       (int)(cw.z & 0xFFFF), (int)(cw.z >> 16), (int)(cw.w & 0xFFFF), (int)(cw.w >> 16)};
  for (int r = 0; r < P.nr; ++r) {
    if (P.sc && *(volatile const int *)&P.sc[r].done) continue;   // uniform over the CTA
    float *R = reinterpret_cast<float *>(vals + (size_t)r * vb);
    // 1. hanging nodes: interpolation of their masters (C)
    for (int j = tid; j < nhang; j += kThreads) {
      const uint2 mw = hent[j];
      const int m0 = mw.x & 0xFFFF, m1 = mw.x >> 16, m2 = mw.y & 0xFFFF, m3 = mw.y >> 16;
      float *d = R + 3 * (nreg + j);
      if (m2 == 0xFFFF) {
#pragma unroll
        for (int c = 0; c < 3; ++c) d[c] = 0.5f * (R[3 * m0 + c] + R[3 * m1 + c]);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          d[c] = 0.25f * ((R[3 * m0 + c] + R[3 * m1 + c]) + (R[3 * m2 + c] + R[3 * m3 + c]));
      }
    }
    __syncthreads();
    // 2. element products into the slot buffer (with the element energies for CG's p^T A p)
    double energy = 0.0;
    if (tid < ne) {
      float X[24], Y[24];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        X[3 * k] = R[3 * code[k]];
        X[3 * k + 1] = R[3 * code[k] + 1];
        X[3 * k + 2] = R[3 * code[k] + 2];
      }
      if (P.sc) energy = (double)element_op<float, kOpBoth>(X, Y, coef, P.K);
      else element_op<float, kOpApply>(X, Y, coef, P.K);
#pragma unroll
      for (int j = 0; j < 24; ++j) XY[tid * kRowM + j] = Y[j];
    }
    if (P.sc) {
      energy = block_sum<kThreads>(energy);
      if (tid == 0) P.dotp[(size_t)r * gridDim.x + b] = energy;
    }
    __syncthreads();
    // 3a. hanging nodes sum their slots
    for (int j = tid; j < nhang; j += kThreads) {
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
      const int q1 = ip[nreg + j + 1];
      for (int q = ip[nreg + j]; q < q1; ++q) {
        const float *d = XY + iv[q];
        s0 += d[0]; s1 += d[1]; s2 += d[2];
      }
      float *h = R + 3 * (nreg + j);
      h[0] = s0; h[1] = s1; h[2] = s2;
    }
    __syncthreads();
    // 3b. regular nodes: slots + folded hanging sums (C^T), then store
    float *y = P.y + (size_t)r * P.ld;
    float *part = P.part + (size_t)r * 3 * P.nslot;
    for (int i = tid; i < nreg; i += kThreads) {
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
      const int q1 = ip[i + 1];
      for (int q = ip[i]; q < q1; ++q) {
        const int p = iv[q];
        if (!(p & kFoldBit)) {
          const float *d = XY + p;
          s0 += d[0]; s1 += d[1]; s2 += d[2];
        } else {
          const float w = (p & kQuarterBit) ? 0.25f : 0.5f;
          const float *h = R + 3 * (nreg + (p & (kQuarterBit - 1)));
          s0 += w * h[0]; s1 += w * h[1]; s2 += w * h[2];
        }
      }
      const uint32_t gw = lnode[i];
      if (gw >> 31) s0 = s1 = s2 = 0.0f;
      float *dst = i < nshared ? part + 3 * (size_t)lslot[i] : y + 3 * (size_t)(gw & 0x7FFFFFFFu);
      dst[0] = s0; dst[1] = s1; dst[2] = s2;
    }
    __syncthreads();   // the slot buffer is reused by the next vector
  }
  }
  // CG: the last CTA sums each running vector's energies: pq = p^T A p, alpha = rz / pq
  if (P.sc && last_cta(P.ticket)) {
    for (int r = 0; r < P.nr; ++r) {
      if (*(volatile const int *)&P.sc[r].done) continue;
      const double pq = sum_partials<kThreads>(P.dotp + (size_t)r * gridDim.x, gridDim.x);
      if (tid == 0) {
        SolveScalars *sc = &P.sc[r];
        sc->pq = pq;
        sc->alpha = sc->rz / pq;
        if (!isfinite(pq) || !isfinite(sc->alpha) || pq <= 0.0) {
          sc->nonfinite = 1;
          sc->done = 1;
        }
      }
      __syncthreads();
    }
  }
}

// Second pass for every vector: shared nodes sum their partials (ascending block
// order); hanging DOFs of y are set to 0.
__global__ void __launch_bounds__(256) shared_multi_kernel(const int32_t *sh_node, const int32_t *sh_ptr, int64_t nsh,
                                                           const int32_t *hang_node, int64_t nh, const float *part,
                                                           int64_t nslot, float *y, int64_t ld, int nr) {
  pdl_begin();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (r >= nr) return;
  const float *pr = part + (size_t)r * 3 * nslot;
  float *yr = y + (size_t)r * ld;
  if (i < nsh) {
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
    for (int j = sh_ptr[i]; j < sh_ptr[i + 1]; ++j) {
      const float *src = pr + 3 * (size_t)j;
      s0 += src[0]; s1 += src[1]; s2 += src[2];
    }
    float *dst = yr + 3 * (size_t)sh_node[i];
    dst[0] = s0; dst[1] = s1; dst[2] = s2;
  } else if (i < nsh + nh) {
    float *dst = yr + 3 * (size_t)hang_node[i - nsh];
    dst[0] = dst[1] = dst[2] = 0.0f;
  }
}

}  // namespace

size_t apply_multi_smem_bytes(const DeviceMesh &m, int nr) {
  const size_t rec_bytes = ((size_t)m.max_rec_bytes + 15) / 16 * 16;
  return std::max(slot_bytes() + (size_t)nr * values_bytes(m.max_local) + rec_bytes, brick_smem_bytes<float>());
}

cudaError_t launch_apply_multi(const DeviceMesh &m, int nr, const float *ce, const float *x, float *y, float *part,
                               double *dotp, SolveScalars *sc, unsigned int *ticket, cudaStream_t s) {
  static std::mutex mu;
  static size_t configured[kStaticMaxDevices] = {};
  const size_t smem = apply_multi_smem_bytes(m, nr);
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kStaticMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (smem > configured[dev]) {
      e = cudaFuncSetAttribute(apply_blocks_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      configured[dev] = smem;
    }
  }
  MultiParams P;
  P.brec = m.brec; P.rec_off = m.rec_off; P.ce = ce; P.x = x; P.y = y; P.part = part;
  P.ld = 3 * m.Nn; P.nslot = m.nslot; P.nr = nr; P.max_local = m.max_local;
  P.dotp = dotp; P.sc = sc; P.ticket = ticket;
  P.nblk = m.nblk;
  P.bricks = BrickTables{m.brick_tab, m.nbrick};
  for (int i = 0; i < 72; ++i) (&P.K.b[0][0][0])[i] = (float)m.modal[i];
  if (apply_ctas(m) > 0) { const cudaError_t pe_ = launch_pdl(apply_blocks_multi_kernel, dim3(apply_ctas(m)), dim3(kThreads), smem, s, P); if (pe_ != cudaSuccess) return pe_; }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || sc) return e;   // inside CG the update kernel sums the partials
  const int64_t items = m.nsh + m.nh;
  const dim3 grid((unsigned)std::max<int64_t>((items + 255) / 256, 1), (unsigned)nr);
  { const cudaError_t pe_ = launch_pdl(shared_multi_kernel, dim3(grid), dim3(256), 0, s, m.sh_node, m.sh_ptr, m.nsh, m.hang_node, m.nh, part, m.nslot, y, 3 * m.Nn,
                                           nr); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}

}  // namespace amr
