// Operator kernels: y = C^T K(rho) C x on the A-space (paper Eq. 6-7), the
// element coefficients c_e = (Emin + rho_e^p (E0 - Emin)) h_e (Eq. 2), the
// Jacobi diagonal of Sec. 5 and the expansion u_full = C u (Eq. 9).
//
// Operator layout (one CTA per block of consecutive elements, tables built by
// mesh_host.cpp).  A block's local nodes are its regular nodes followed by the
// hanging nodes its elements use; each local node has an inverse list of the
// (element, corner) slots it fills.
//   1. regular nodes load x (Dirichlet entries read as 0) and write it into
//      their slots of a per-element shared buffer; hanging nodes then write the
//      (bi)linear interpolation of their masters into theirs (C, Eq. 6);
//   2. one thread per element replaces its 24 inputs by c_e K0 X_e (sum
//      factorisation, element.cuh);
//   3. hanging nodes sum their slots; regular nodes sum their slots plus
//      w * (sum) of every hanging node they are a master of (C^T) -- a fixed
//      summation order, no atomics, bitwise reproducible;
//   4. nodes touched only by this block are stored to y; nodes shared with
//      other blocks are stored to per-block slots that a second kernel sums in
//      ascending block order.  Hanging DOFs of y are set to 0.
// The dot product x . y can be accumulated on the fly (CG's p^T A p).
#include <cuda_runtime.h>

#include "element.cuh"
#include "pcg.cuh"
#include "reduce.cuh"
#include "tm_internal.h"

namespace amr {

constexpr int kApplyThreads = kBlockElems;  // one thread per element of a block
constexpr int kRow = 25;                    // padded per-element row of the slot buffer

template <typename T>
struct ApplyParams {
  const int32_t *blk_elem, *blk_node, *blk_shared, *blk_slot, *blk_hang, *blk_iptr, *blk_inv;
  const int32_t *lnode, *lslot;
  const uint16_t *hent, *iptr, *inv;
  const uint8_t *nflag;
  const T *ce;
  const T *x;
  T *y;
  T *part;
  double *dotp;     // per-CTA partials of x . y (nullptr: skip)
  const int *done;  // skip the launch when set (nullptr: never)
  T lam, mu;
};

template <typename T>
size_t apply_smem_bytes(int max_local) {
  return sizeof(T) * ((size_t)kApplyThreads * kRow + 3 * (size_t)max_local);
}

__device__ __forceinline__ int slot_of(int p) { return (p >> 3) * kRow + 3 * (p & 7); }

template <typename T>
__global__ void __launch_bounds__(kApplyThreads, sizeof(T) == 4 ? 4 : 2) apply_blocks_kernel(ApplyParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *XY = reinterpret_cast<T *>(smem_raw);   // per-element slots: inputs, then outputs
  T *R = XY + kApplyThreads * kRow;          // regular x values, then hanging sums

  if (P.done && *(volatile const int *)P.done) return;
  const int b = blockIdx.x;
  const int tid = threadIdx.x;
  const int e0 = P.blk_elem[b], ne = P.blk_elem[b + 1] - e0;
  const int n0 = P.blk_node[b], nreg = P.blk_node[b + 1] - n0;
  const int h0 = P.blk_hang[b], nhang = P.blk_hang[b + 1] - h0;
  const uint16_t *ip = P.iptr + P.blk_iptr[b];
  const uint16_t *iv = P.inv + P.blk_inv[b];

  // 1a. regular nodes: load and scatter into their slots
  for (int i = tid; i < nreg; i += kApplyThreads) {
    const int g = P.lnode[n0 + i];
    const bool fixed = P.nflag[g] & 1;
    const T *src = P.x + 3 * (size_t)g;
    const T v0 = fixed ? T(0) : src[0], v1 = fixed ? T(0) : src[1], v2 = fixed ? T(0) : src[2];
    R[3 * i] = v0; R[3 * i + 1] = v1; R[3 * i + 2] = v2;
    const int q1 = ip[i + 1];
    for (int q = ip[i]; q < q1; ++q) {
      const int p = iv[q];
      if (p & kFoldBit) continue;
      T *d = XY + slot_of(p);
      d[0] = v0; d[1] = v1; d[2] = v2;
    }
  }
  __syncthreads();
  // 1b. hanging nodes: interpolate the masters (C) and scatter
  for (int j = tid; j < nhang; j += kApplyThreads) {
    const uint2 mw = reinterpret_cast<const uint2 *>(P.hent)[h0 + j];
    const int m0 = mw.x & 0xFFFF, m1 = mw.x >> 16, m2 = mw.y & 0xFFFF, m3 = mw.y >> 16;
    T v[3];
    if (m2 == 0xFFFF) {
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] = T(0.5) * (R[3 * m0 + c] + R[3 * m1 + c]);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] = T(0.25) * ((R[3 * m0 + c] + R[3 * m1 + c]) + (R[3 * m2 + c] + R[3 * m3 + c]));
    }
    const int q1 = ip[nreg + j + 1];
    for (int q = ip[nreg + j]; q < q1; ++q) {
      T *d = XY + slot_of(iv[q]);
      d[0] = v[0]; d[1] = v[1]; d[2] = v[2];
    }
  }
  __syncthreads();
  // 2. element operator, in place
  if (tid < ne) {
    T X[24], Y[24];
#pragma unroll
    for (int j = 0; j < 24; ++j) X[j] = XY[tid * kRow + j];
    element_op<T, false>(X, Y, P.ce[e0 + tid], P.lam, P.mu);
#pragma unroll
    for (int j = 0; j < 24; ++j) XY[tid * kRow + j] = Y[j];
  }
  __syncthreads();
  // 3a. hanging nodes sum their slots
  for (int j = tid; j < nhang; j += kApplyThreads) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    const int q1 = ip[nreg + j + 1];
    for (int q = ip[nreg + j]; q < q1; ++q) {
      const T *d = XY + slot_of(iv[q]);
      s0 += d[0]; s1 += d[1]; s2 += d[2];
    }
    T *r = R + 3 * (nreg + j);
    r[0] = s0; r[1] = s1; r[2] = s2;
  }
  __syncthreads();
  // 3b/4. regular nodes: own slots + folded hanging sums (C^T), then store
  const int nshared = P.blk_shared[b];
  const int slot0 = P.blk_slot[b];
  double dot = 0.0;
  for (int i = tid; i < nreg; i += kApplyThreads) {
    T s0 = T(0), s1 = T(0), s2 = T(0);
    const int q1 = ip[i + 1];
    for (int q = ip[i]; q < q1; ++q) {
      const int p = iv[q];
      if (!(p & kFoldBit)) {
        const T *d = XY + slot_of(p);
        s0 += d[0]; s1 += d[1]; s2 += d[2];
      } else {
        const T w = (p & kQuarterBit) ? T(0.25) : T(0.5);
        const T *r = R + 3 * (nreg + (p & (kQuarterBit - 1)));
        s0 += w * r[0]; s1 += w * r[1]; s2 += w * r[2];
      }
    }
    const int g = P.lnode[n0 + i];
    if (P.nflag[g] & 1) s0 = s1 = s2 = T(0);
    if (i < nshared) {
      T *dst = P.part + 3 * (size_t)P.lslot[slot0 + i];
      dst[0] = s0; dst[1] = s1; dst[2] = s2;
    } else {
      T *dst = P.y + 3 * (size_t)g;
      dst[0] = s0; dst[1] = s1; dst[2] = s2;
      dot += (double)R[3 * i] * (double)s0 + (double)R[3 * i + 1] * (double)s1 + (double)R[3 * i + 2] * (double)s2;
    }
  }
  if (P.dotp) {
    dot = block_sum<kApplyThreads>(dot);
    if (tid == 0) P.dotp[b] = dot;
  }
}

// Second pass: each shared node sums its contiguous run of partials (one per
// block touching it, in ascending block order); optionally hanging DOFs of y are
// zeroed.  With dot partials, the last CTA also finishes p^T A p and sets
// alpha = rz / pq for CG (when sc is given).
template <typename T>
__global__ void __launch_bounds__(256) apply_shared_kernel(const int32_t *sh_node, const int32_t *sh_ptr, int64_t nsh,
                                                           const int32_t *hang_node, int64_t nh,
                                                           const uint8_t *nflag, const T *part, const T *x,
                                                           T *y, double *dotp, int nblk_partials,
                                                           SolveScalars *sc, unsigned int *ticket,
                                                           const int *done) {
  if (done && *(volatile const int *)done) return;
  double dot = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nsh + nh;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nsh) {
      const int g = sh_node[i];
      T s0 = T(0), s1 = T(0), s2 = T(0);
      for (int j = sh_ptr[i]; j < sh_ptr[i + 1]; ++j) {
        const T *src = part + 3 * (size_t)j;
        s0 += src[0]; s1 += src[1]; s2 += src[2];
      }
      T *dst = y + 3 * (size_t)g;
      dst[0] = s0; dst[1] = s1; dst[2] = s2;
      if (dotp) {
        const T *xv = x + 3 * (size_t)g;
        if (!(nflag[g] & 1))
          dot += (double)xv[0] * (double)s0 + (double)xv[1] * (double)s1 + (double)xv[2] * (double)s2;
      }
    } else {
      T *dst = y + 3 * (size_t)hang_node[i - nsh];
      dst[0] = dst[1] = dst[2] = T(0);
    }
  }
  if (dotp) {
    dot = block_sum<256>(dot);
    if (threadIdx.x == 0) dotp[nblk_partials + blockIdx.x] = dot;
    if (sc && last_cta(ticket)) {
      const double pq = sum_partials<256>(dotp, nblk_partials + gridDim.x);
      if (threadIdx.x == 0) {
        sc->pq = pq;
        sc->alpha = sc->rz / pq;
        if (!isfinite(pq) || !isfinite(sc->alpha) || pq <= 0.0) {
          sc->nonfinite = 1;
          sc->done = 1;
        }
      }
    }
  }
}

int shared_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 1216) g = 1216;  // 8 CTAs per SM on 152 SMs; grid-stride beyond
  return (int)g;
}

template <typename T>
cudaError_t launch_apply(const DeviceMesh &m, const T *ce, const T *x, T *y, T *part, double *dot_partials,
                         SolveScalars *sc, unsigned int *ticket, bool zero_hanging, const int *done,
                         cudaStream_t s) {
  static size_t configured = 0;
  const size_t smem = apply_smem_bytes<T>(m.max_local);
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(apply_blocks_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)apply_smem_bytes<T>(kMaxLocal));
    if (e != cudaSuccess) return e;
    configured = apply_smem_bytes<T>(kMaxLocal);
  }
  ApplyParams<T> P;
  P.blk_elem = m.blk_elem; P.blk_node = m.blk_node; P.blk_shared = m.blk_shared; P.blk_slot = m.blk_slot;
  P.blk_hang = m.blk_hang; P.blk_iptr = m.blk_iptr; P.blk_inv = m.blk_inv; P.lnode = m.lnode; P.lslot = m.lslot;
  P.hent = m.hent; P.iptr = m.iptr; P.inv = m.inv; P.nflag = m.nflag; P.ce = ce; P.x = x; P.y = y; P.part = part;
  P.dotp = dot_partials; P.done = done; P.lam = (T)m.lam; P.mu = (T)m.mu;
  if (m.nblk > 0) apply_blocks_kernel<T><<<m.nblk, kApplyThreads, smem, s>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t items = m.nsh + (zero_hanging ? m.nh : 0);
  apply_shared_kernel<T><<<shared_grid(items), 256, 0, s>>>(m.sh_node, m.sh_ptr, m.nsh, m.hang_node,
                                                            zero_hanging ? m.nh : 0, m.nflag, part, x, y,
                                                            dot_partials, m.nblk, sc, ticket, done);
  return cudaGetLastError();
}

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

cudaError_t static_scratch(int device, float **ce, float **part) {
  if (device < 0 || device >= kStaticMaxDevices) return cudaErrorInvalidDevice;
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
