// Fused vector kernels of Jacobi-preconditioned CG (paper Sec. 5: the diagonal
// rescaling D^-1/2 K D^-1/2 applied implicitly as the preconditioner) with FP64
// reductions finalised on the device, so the iteration needs no host round trip.
//
// Iteration (x: solution, z = Dinv r is never stored):
//   q = A p ; pq = sum of element energies of p, alpha = rz / pq (in the operator's
//   block pass; the q of shared nodes is summed from their partials by the update)
//   x += alpha p ; r -= alpha q ; rz' = r.Dinv r ; rr = r.r          beta = rz' / rz
//   p = Dinv r + beta p
// Every kernel returns immediately once the device flag `done` is set, so a
// fixed batch of iterations can be enqueued (or graph-captured) ahead of the
// host's convergence check.
#include <cuda_runtime.h>

#include "pcg.cuh"
#include "pdl.cuh"
#include "reduce.cuh"
#include "tm_internal.h"

namespace amr {

constexpr int kVecThreads = 256;

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

template <typename TX, typename T>
__global__ void __launch_bounds__(kVecThreads) update_kernel(TX *x, const T *p, const T *q, T *r, const T *dinv,
                                                             int64_t n, SolveScalars *sc, double *partials,
                                                             unsigned int *ticket) {
  pdl_begin();
  if (sc->done) return;
  const double alpha = sc->alpha;
  const T a = (T)alpha;
  DotAcc<T> arz, arr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += (TX)alpha * (TX)p[i];
    const T ri = r[i] - a * q[i];
    r[i] = ri;
    arz.add_prod(ri, dinv[i] * ri);
    arr.add_prod(ri, ri);
  }
  double rz = arz.value(), rr = arr.value();
  block_sum2<kVecThreads>(rz, rr);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = rz;
    partials[2 * blockIdx.x + 1] = rr;
  }
  if (last_cta(ticket)) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kVecThreads) {
      s0 += ((volatile double *)partials)[2 * i];
      s1 += ((volatile double *)partials)[2 * i + 1];
    }
    block_sum2<kVecThreads>(s0, s1);
    if (threadIdx.x == 0) {
      sc->beta = s0 / sc->rz;
      sc->rz_prev = sc->rz;
      sc->rz = s0;
      sc->rr = s1;
      sc->it += 1;
      if (s1 > sc->rrmax) sc->rrmax = s1;
      if (!finite(s0) || !finite(s1)) {
        sc->nonfinite = 1;
        sc->done = 1;
      } else if (s1 <= fmax(sc->stop_ratio2 * sc->rrmax, sc->stop_abs_rr) || sc->it >= sc->max_it) {
        sc->done = 1;
        sc->last_beta_skipped = 1;
      }
    }
  }
}

// Same update, node by node, for an operator result q that is complete only at
// nodes owned by one block: the q of a shared node is the sum of its partials
// (contiguous, ascending block order), read here instead of a second pass.
template <typename TX, typename T>
__global__ void __launch_bounds__(kVecThreads) update_nodes_kernel(TX *x, const T *p, const T *q, T *r, const T *dinv,
                                                                   int64_t Nn, const int32_t *sh_of_node,
                                                                   const int32_t *sh_ptr, const T *part,
                                                                   SolveScalars *sc, double *partials,
                                                                   unsigned int *ticket, int twolevel, int64_t vst,
                                                                   int64_t pst, int pstride) {
  pdl_begin();
  // load case blockIdx.y: its vectors vst apart, its partial sums pst apart, its own scalars,
  // reduction partials and ticket
  const int cs = blockIdx.y;
  sc += cs;
  if (sc->done) return;
  x += cs * vst; p += cs * vst; q += cs * vst; r += cs * vst;
  part += cs * pst;
  partials += (int64_t)cs * pstride;
  ticket += cs;
  const double alpha = sc->alpha;
  const T a = (T)alpha;
  DotAcc<T> arz, arr;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < Nn; n += (int64_t)gridDim.x * blockDim.x) {
    T qv[3];
    const int sh = sh_of_node[n];
    if (sh < 0) {
      qv[0] = q[3 * n]; qv[1] = q[3 * n + 1]; qv[2] = q[3 * n + 2];
    } else {
      qv[0] = qv[1] = qv[2] = T(0);
      for (int j = sh_ptr[sh]; j < sh_ptr[sh + 1]; ++j) {
        qv[0] += part[3 * (size_t)j]; qv[1] += part[3 * (size_t)j + 1]; qv[2] += part[3 * (size_t)j + 2];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t i = 3 * n + c;
      x[i] += (TX)alpha * (TX)p[i];
      const T ri = r[i] - a * qv[c];
      r[i] = ri;
      arz.add_prod(ri, dinv[i] * ri);
      arr.add_prod(ri, ri);
    }
  }
  double rz = arz.value(), rr = arr.value();
  block_sum2<kVecThreads>(rz, rr);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = rz;
    partials[2 * blockIdx.x + 1] = rr;
  }
  if (last_cta(ticket)) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kVecThreads) {
      s0 += ((volatile double *)partials)[2 * i];
      s1 += ((volatile double *)partials)[2 * i + 1];
    }
    block_sum2<kVecThreads>(s0, s1);
    if (threadIdx.x == 0) {
      if (twolevel) {
        sc->scratch[0] = s0;     // r^T D^-1 r; the coarse term and beta follow (kernels_coarse.cu)
        sc->rz_prev = sc->rz;    // the rz the current p was built from (a residual replacement needs it)
      } else {
        sc->beta = s0 / sc->rz;
        sc->rz_prev = sc->rz;
        sc->rz = s0;
      }
      sc->rr = s1;
      sc->it += 1;
      if (s1 > sc->rrmax) sc->rrmax = s1;
      if (!finite(s0) || !finite(s1)) {
        sc->nonfinite = 1;
        sc->done = 1;
      } else if (s1 <= fmax(sc->stop_ratio2 * sc->rrmax, sc->stop_abs_rr) || sc->it >= sc->max_it) {
        sc->done = 1;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kVecThreads) pupdate_kernel(T *p, const T *r, const T *dinv, int64_t n,
                                                              SolveScalars *sc) {
  pdl_begin();
  if (sc->done) return;
  const T beta = (T)sc->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = dinv[i] * r[i] + beta * p[i];
}

// r = s * (f - q) (q = A x0); p = Dinv r; rz, rr; stop threshold from rr0.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) start_kernel(const double *f, const double *q, double scale, T *r,
                                                            T *p, const T *dinv, int64_t n, SolveScalars *sc,
                                                            double *partials, unsigned int *ticket) {
  DotAcc<T> arz, arr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = (T)(scale * (f[i] - (q ? q[i] : 0.0)));
    r[i] = ri;
    const T zi = dinv[i] * ri;
    p[i] = zi;
    arz.add_prod(ri, zi);
    arr.add_prod(ri, ri);
  }
  double rz = arz.value(), rr = arr.value();
  block_sum2<kVecThreads>(rz, rr);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = rz;
    partials[2 * blockIdx.x + 1] = rr;
  }
  if (last_cta(ticket)) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kVecThreads) {
      s0 += ((volatile double *)partials)[2 * i];
      s1 += ((volatile double *)partials)[2 * i + 1];
    }
    block_sum2<kVecThreads>(s0, s1);
    if (threadIdx.x == 0) {
      sc->rz = s0;
      sc->rr = s1;
      sc->rr0 = s1;
      sc->rrmax = s1;
      sc->it = 0;
      sc->nonfinite = 0;
      sc->last_beta_skipped = 0;
      sc->stop_rr = sc->stop_ratio2 * s1;
      if (sc->stop_abs_rr > sc->stop_rr) sc->stop_rr = sc->stop_abs_rr;
      sc->done = (s1 <= sc->stop_rr || s1 == 0.0) ? 1 : 0;
      if (!finite(s0) || !finite(s1)) {
        sc->nonfinite = 1;
        sc->done = 1;
      }
    }
  }
}

// r64 = f - q; rr = r.r (FP64): the true residual of the mixed solver's reliable updates.
__global__ void __launch_bounds__(kVecThreads) residual64_kernel(const double *f, const double *q, double *r,
                                                                 int64_t n, double *out, double *partials,
                                                                 unsigned int *ticket) {
  double rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = f[i] - (q ? q[i] : 0.0);
    if (r) r[i] = ri;
    rr += ri * ri;
  }
  rr = block_sum<kVecThreads>(rr);
  if (threadIdx.x == 0) partials[blockIdx.x] = rr;
  if (last_cta(ticket)) {
    const double s = sum_partials<kVecThreads>(partials, gridDim.x);
    if (threadIdx.x == 0) *out = s;
  }
}

// u += s * d (FP64 accumulate of an FP32 correction); d is cleared.
__global__ void correct_kernel(double *u, float *d, double s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    u[i] += s * (double)d[i];
    d[i] = 0.0f;
  }
}

// Residual replacement, pass 1: r = scale * r64, p *= c; rz = r.Dinv r, rp = r.p,
// rr = r.r.  The last CTA sets beta = rz / (rz_prev c^2) (the previous iteration's
// rz in the new units) and gamma = rp / rz, and restarts the run's counters.
__global__ void __launch_bounds__(kVecThreads) replace_dots_kernel(const double *r64, double scale, double c, float *r,
                                                                   float *p, const float *dinv, int64_t n,
                                                                   double stop_abs_rr, int max_it, SolveScalars *sc,
                                                                   double *partials, unsigned int *ticket) {
  DotAcc<float> arz, arp, arr;
  const float cf = (float)c;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float ri = (float)(scale * r64[i]);
    const float pi = p[i] * cf;
    r[i] = ri;
    p[i] = pi;
    arz.add_prod(ri, dinv[i] * ri);
    arp.add_prod(ri, pi);
    arr.add_prod(ri, ri);
  }
  double rz = arz.value(), rp = arp.value(), rr = arr.value();
  block_sum2<kVecThreads>(rz, rp);
  rr = block_sum<kVecThreads>(rr);
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = rz;
    partials[3 * blockIdx.x + 1] = rp;
    partials[3 * blockIdx.x + 2] = rr;
  }
  if (last_cta(ticket)) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kVecThreads) {
      s0 += ((volatile double *)partials)[3 * i];
      s1 += ((volatile double *)partials)[3 * i + 1];
      s2 += ((volatile double *)partials)[3 * i + 2];
    }
    block_sum2<kVecThreads>(s0, s1);
    s2 = block_sum<kVecThreads>(s2);
    if (threadIdx.x == 0) {
      const double prev = sc->rz_prev * c * c;
      sc->beta = s0 / prev;
      sc->rp = s1 / s0;        // gamma
      sc->scratch[2] = prev;   // kept for the two-level preconditioner's beta and gamma
      sc->scratch[3] = s1;
      sc->rz = s0;
      sc->rr = s2;
      sc->rr0 = s2;
      sc->rrmax = s2;
      sc->it = 0;
      sc->max_it = max_it;
      sc->stop_abs_rr = stop_abs_rr;
      sc->nonfinite = 0;
      sc->last_beta_skipped = 0;
      sc->done = (s2 <= stop_abs_rr || s2 == 0.0) ? 1 : 0;
      if (!finite(s0) || !finite(s1) || !finite(s2) || !finite(sc->beta) || s0 <= 0.0) {
        sc->nonfinite = 1;
        sc->done = 1;
      }
    }
  }
}

// Pass 2: p = z + beta (p - gamma z) with z = Dinv r.
__global__ void __launch_bounds__(kVecThreads) replace_p_kernel(const float *r, float *p, const float *dinv, int64_t n,
                                                                const SolveScalars *sc) {
  if (sc->done) return;
  const float beta = (float)sc->beta, gamma = (float)sc->rp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float zi = dinv[i] * r[i];
    p[i] = zi + beta * (p[i] - gamma * zi);
  }
}

__global__ void mask_kernel(const uint8_t *nflag, double *u, int64_t Nn) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Nn; k += (int64_t)gridDim.x * blockDim.x)
    if (nflag[k]) u[3 * k] = u[3 * k + 1] = u[3 * k + 2] = 0.0;
}

int vec_grid(int64_t n) {
  int64_t g = (n + kVecThreads - 1) / kVecThreads;
  if (g < 1) g = 1;
  if (g > 8 * device_sms()) g = 8 * device_sms();
  return (int)g;
}

template <typename TX, typename T>
cudaError_t launch_update(TX *x, const T *p, const T *q, T *r, const T *dinv, int64_t n, SolveScalars *sc,
                          double *partials, unsigned int *ticket, cudaStream_t s) {
  { const cudaError_t pe_ = launch_pdl(update_kernel<TX, T>, dim3(vec_grid(n)), dim3(kVecThreads), 0, s, x, p, q, r, dinv, n, sc, partials, ticket); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}
template cudaError_t launch_update<double, double>(double *, const double *, const double *, double *,
                                                   const double *, int64_t, SolveScalars *, double *,
                                                   unsigned int *, cudaStream_t);
template cudaError_t launch_update<float, float>(float *, const float *, const float *, float *, const float *,
                                                 int64_t, SolveScalars *, double *, unsigned int *, cudaStream_t);

template <typename TX, typename T>
cudaError_t launch_update_nodes(TX *x, const T *p, const T *q, T *r, const T *dinv, int64_t Nn,
                                const int32_t *sh_of_node, const int32_t *sh_ptr, const T *part, SolveScalars *sc,
                                double *partials, unsigned int *ticket, cudaStream_t s, bool twolevel) {
  { const cudaError_t pe_ = launch_pdl(update_nodes_kernel<TX, T>, dim3(vec_grid(Nn)), dim3(kVecThreads), 0, s, x, p, q, r, dinv, Nn, sh_of_node, sh_ptr, part, sc,
                                                                   partials, ticket, twolevel ? 1 : 0, 0, 0, 0); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}
template cudaError_t launch_update_nodes<double, double>(double *, const double *, const double *, double *,
                                                         const double *, int64_t, const int32_t *, const int32_t *,
                                                         const double *, SolveScalars *, double *, unsigned int *,
                                                         cudaStream_t, bool);
template cudaError_t launch_update_nodes<float, float>(float *, const float *, const float *, float *, const float *,
                                                       int64_t, const int32_t *, const int32_t *, const float *,
                                                       SolveScalars *, double *, unsigned int *, cudaStream_t, bool);

cudaError_t launch_update_nodes_cases(int nv, float *x, const float *p, const float *q, float *r, int64_t vst,
                                      const float *dinv, int64_t Nn, const int32_t *sh_of_node, const int32_t *sh_ptr,
                                      const float *part, int64_t pst, SolveScalars *sc, double *partials,
                                      unsigned int *tickets, cudaStream_t s, bool twolevel) {
  const int g = vec_grid(Nn);
  { const cudaError_t pe_ = launch_pdl(update_nodes_kernel<float, float>, dim3(dim3(g, nv)), dim3(kVecThreads), 0, s, x, p, q, r, dinv, Nn, sh_of_node, sh_ptr, part,
                                                                        sc, partials, tickets, twolevel ? 1 : 0, vst,
                                                                        pst, 2 * g); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pupdate(T *p, const T *r, const T *dinv, int64_t n, SolveScalars *sc, cudaStream_t s) {
  { const cudaError_t pe_ = launch_pdl(pupdate_kernel<T>, dim3(vec_grid(n)), dim3(kVecThreads), 0, s, p, r, dinv, n, sc); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}
template cudaError_t launch_pupdate<double>(double *, const double *, const double *, int64_t, SolveScalars *,
                                            cudaStream_t);
template cudaError_t launch_pupdate<float>(float *, const float *, const float *, int64_t, SolveScalars *,
                                           cudaStream_t);

template <typename T>
cudaError_t launch_start(const double *f, const double *q, double scale, T *r, T *p, const T *dinv, int64_t n,
                         SolveScalars *sc, double *partials, unsigned int *ticket, cudaStream_t s) {
  start_kernel<T><<<vec_grid(n), kVecThreads, 0, s>>>(f, q, scale, r, p, dinv, n, sc, partials, ticket);
  return cudaGetLastError();
}
template cudaError_t launch_start<double>(const double *, const double *, double, double *, double *,
                                          const double *, int64_t, SolveScalars *, double *, unsigned int *,
                                          cudaStream_t);
template cudaError_t launch_start<float>(const double *, const double *, double, float *, float *, const float *,
                                         int64_t, SolveScalars *, double *, unsigned int *, cudaStream_t);

cudaError_t launch_residual64(const double *f, const double *q, double *r, int64_t n, double *out, double *partials,
                              unsigned int *ticket, cudaStream_t s) {
  residual64_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(f, q, r, n, out, partials, ticket);
  return cudaGetLastError();
}

cudaError_t launch_replace(const double *r64, double scale, double c, float *r, float *p, const float *dinv,
                           int64_t n, double stop_abs_rr, int max_it, SolveScalars *sc, double *partials,
                           unsigned int *ticket, cudaStream_t s, bool dots_only) {
  replace_dots_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(r64, scale, c, r, p, dinv, n, stop_abs_rr, max_it, sc,
                                                          partials, ticket);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || dots_only) return e;
  replace_p_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(r, p, dinv, n, sc);
  return cudaGetLastError();
}

cudaError_t launch_correct(double *u, float *d, double scale, int64_t n, cudaStream_t s) {
  correct_kernel<<<vec_grid(n), kVecThreads, 0, s>>>(u, d, scale, n);
  return cudaGetLastError();
}

cudaError_t launch_mask(const uint8_t *nflag, double *u, int64_t Nn, cudaStream_t s) {
  mask_kernel<<<vec_grid(Nn), kVecThreads, 0, s>>>(nflag, u, Nn);
  return cudaGetLastError();
}

}  // namespace amr
