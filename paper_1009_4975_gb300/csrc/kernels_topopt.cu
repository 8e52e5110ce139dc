// Optimisation-step kernels: compliance sensitivities (paper Sec. 3), the
// filters of Eq. 3-5, and the optimality-criteria update with a device-side
// bisection on the Lagrange multiplier of the volume constraint.
#include <cuda_runtime.h>

#include "element.cuh"
#include "reduce.cuh"
#include "tm_internal.h"
#include "topopt.cuh"

namespace amr {

constexpr int kTopThreads = 256;

// dc_e = -p rho^(p-1) (E0 - Emin) h_e u_e^T K0 u_e ; compliance partial E_e h_e u_e^T K0 u_e.
__global__ void __launch_bounds__(kTopThreads) sensitivity_kernel(const int32_t *conn, const int32_t *leaf,
                                                                  const double *rho, const double *uf, int64_t Ne,
                                                                  double E0, double Emin, double penal, double h0,
                                                                  ModalBlocks<double> K, double *dc,
                                                                  double *partials, unsigned int *ticket,
                                                                  double *compliance) {
  double cpart = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    double X[24];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double *src = uf + 3 * (size_t)conn[8 * e + k];
      X[3 * k] = src[0];
      X[3 * k + 1] = src[1];
      X[3 * k + 2] = src[2];
    }
    const double en = element_op<double, kOpEnergy>(X, nullptr, 1.0, K);
    const double h = ldexp(h0, -leaf[4 * e + 3]);
    const double r = rho[e];
    dc[e] = -penal * pow(r, penal - 1.0) * (E0 - Emin) * h * en;
    cpart += (Emin + pow(r, penal) * (E0 - Emin)) * h * en;
  }
  cpart = block_sum<kTopThreads>(cpart);
  if (threadIdx.x == 0) partials[blockIdx.x] = cpart;
  if (last_cta(ticket)) {
    const double s = sum_partials<kTopThreads>(partials, gridDim.x);
    if (threadIdx.x == 0) *compliance = s;
  }
}

int top_grid(int64_t n) {
  int64_t g = (n + kTopThreads - 1) / kTopThreads;
  if (g < 1) g = 1;
  if (g > 8 * device_sms()) g = 8 * device_sms();
  return (int)g;
}

cudaError_t launch_sensitivity(const DeviceMesh &m, const double *rho, const double *uf, double *dc,
                               double *partials, unsigned int *ticket, double *compliance, cudaStream_t s) {
  ModalBlocks<double> K;
  for (int i = 0; i < 72; ++i) (&K.b[0][0][0])[i] = m.modal[i];
  sensitivity_kernel<<<top_grid(m.Ne), kTopThreads, 0, s>>>(m.conn, m.leaf, rho, uf, m.Ne, m.E0, m.Emin, m.penal,
                                                            m.h0, K, dc, partials, ticket, compliance);
  return cudaGetLastError();
}

// For element e: every element d whose centre lies within rmin of e's centre,
// found through the finest-cell map over the box [c - rmin, c + rmin].  A leaf
// covering several cells of the box is taken once, at its first cell in scan
// order (the componentwise max of its anchor and the box's low corner).
__global__ void __launch_bounds__(kTopThreads) filter_kernel(const int32_t *leaf, const int32_t *cellmap, int fx,
                                                             int fy, int fz, int L, double unit, const double *rho,
                                                             const double *x, double rmin, int mode, int64_t Ne,
                                                             double *out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    const int *le = leaf + 4 * e;
    const int se = 1 << (L - le[3]);
    // centre in finest units (exact in double)
    const double cx = le[0] + 0.5 * se, cy = le[1] + 0.5 * se, cz = le[2] + 0.5 * se;
    const double ru = rmin / unit;
    int lo[3], hi[3];
    const double c[3] = {cx, cy, cz};
    const int ext[3] = {fx, fy, fz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // cells i with i < c + ru and i + 1 > c - ru
      lo[a] = (int)floor(c[a] - ru);
      hi[a] = (int)ceil(c[a] + ru) - 1;
      if (lo[a] < 0) lo[a] = 0;
      if (hi[a] > ext[a] - 1) hi[a] = ext[a] - 1;
    }
    double num = 0.0, den = 0.0;
    for (int iz = lo[2]; iz <= hi[2]; ++iz)
      for (int iy = lo[1]; iy <= hi[1]; ++iy)
        for (int ix = lo[0]; ix <= hi[0]; ++ix) {
          const int d = cellmap[((size_t)iz * fy + iy) * fx + ix];
          const int *ld = leaf + 4 * d;
          const int fxd = ld[0] > lo[0] ? ld[0] : lo[0];
          const int fyd = ld[1] > lo[1] ? ld[1] : lo[1];
          const int fzd = ld[2] > lo[2] ? ld[2] : lo[2];
          if (ix != fxd || iy != fyd || iz != fzd) continue;
          const int sd = 1 << (L - ld[3]);
          const double dx = (ld[0] + 0.5 * sd - cx) * unit, dy = (ld[1] + 0.5 * sd - cy) * unit,
                       dz = (ld[2] + 0.5 * sd - cz) * unit;
          const double dist = sqrt(dx * dx + dy * dy + dz * dz);
          if (!(dist < rmin)) continue;
          const double hd = sd * unit;
          const double w = (rmin - dist) * hd * hd * hd;
          num += mode == 0 ? w * rho[d] * x[d] : w * x[d];
          den += w;
        }
    out[e] = mode == 0 ? num / (rho[e] * den) : num / den;
  }
}

cudaError_t launch_filter(const DeviceMesh &m, const double *rho, const double *x, double rmin, int mode,
                          double *out, cudaStream_t s) {
  filter_kernel<<<top_grid(m.Ne), kTopThreads, 0, s>>>(m.leaf, m.cellmap, m.fx, m.fy, m.fz, m.L, m.hmin, rho, x, rmin,
                                                       mode, m.Ne, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- OC
// OcState lives in device memory; the bisection runs as a fixed number of
// launches of oc_volume_kernel, each of which evaluates sum rho_new(lambda) V_e at
// the bracket midpoint and narrows the bracket in its last CTA.  Once the
// relative bracket is below tol the remaining launches return at once.
__device__ __forceinline__ double oc_value(double r, double g, double V, double lam, double eta, double move,
                                           double rmin) {
  const double lo = fmax(rmin, r - move), hi = fmin(1.0, r + move);
  const double t = g / (lam * V);
  const double v = r * (eta == 0.5 ? sqrt(t) : pow(t, eta));
  return fmin(fmax(v, lo), hi);
}

__global__ void __launch_bounds__(kTopThreads) oc_init_kernel(const int32_t *leaf, const double *dc, int64_t Ne,
                                                              int L, double h0, double *partials,
                                                              unsigned int *ticket, OcState *st) {
  double gmax = 0.0, vmin = 1e300;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    const double g = fmax(-dc[e], 0.0);
    const double h = ldexp(h0, -leaf[4 * e + 3]);
    gmax = fmax(gmax, g);
    vmin = fmin(vmin, h * h * h);
  }
  // max / min through negated sums is not possible; use a shared-memory tree
  __shared__ double sm[kTopThreads], sv[kTopThreads];
  sm[threadIdx.x] = gmax;
  sv[threadIdx.x] = vmin;
  __syncthreads();
  for (int o = kTopThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
      sv[threadIdx.x] = fmin(sv[threadIdx.x], sv[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sm[0];
    partials[2 * blockIdx.x + 1] = sv[0];
  }
  if (last_cta(ticket)) {
    if (threadIdx.x == 0) {
      double a = 0.0, b = 1e300;
      for (int i = 0; i < (int)gridDim.x; ++i) {
        a = fmax(a, ((volatile double *)partials)[2 * i]);
        b = fmin(b, ((volatile double *)partials)[2 * i + 1]);
      }
      st->l1 = 0.0;
      st->l2 = 1e9 * fmax(a, 1e-300) / b;
      st->done = 0;
      st->iters = 0;
    }
  }
}

__global__ void __launch_bounds__(kTopThreads) oc_volume_kernel(const int32_t *leaf, const double *rho,
                                                                const double *dc, int64_t Ne, int L, double h0,
                                                                double eta, double move, double rmin,
                                                                double *partials, unsigned int *ticket,
                                                                OcState *st) {
  if (st->done) return;
  const double lam = 0.5 * (st->l1 + st->l2);
  double vol = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    const double h = ldexp(h0, -leaf[4 * e + 3]);
    const double V = h * h * h;
    vol += oc_value(rho[e], fmax(-dc[e], 0.0), V, lam, eta, move, rmin) * V;
  }
  vol = block_sum<kTopThreads>(vol);
  if (threadIdx.x == 0) partials[blockIdx.x] = vol;
  if (last_cta(ticket)) {
    const double s = sum_partials<kTopThreads>(partials, gridDim.x);
    if (threadIdx.x == 0) {
      if (s > st->target) st->l1 = lam;
      else st->l2 = lam;
      st->iters += 1;
      if (st->l2 - st->l1 <= st->tol * (st->l1 + st->l2)) st->done = 1;
    }
  }
}

__global__ void __launch_bounds__(kTopThreads) oc_final_kernel(const int32_t *leaf, const double *rho,
                                                               const double *dc, int64_t Ne, int L, double h0,
                                                               double eta, double move, double rmin,
                                                               double *rho_new, double *partials,
                                                               unsigned int *ticket, OcState *st) {
  const double lam = 0.5 * (st->l1 + st->l2);
  double chg = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    const double h = ldexp(h0, -leaf[4 * e + 3]);
    const double V = h * h * h;
    const double v = oc_value(rho[e], fmax(-dc[e], 0.0), V, lam, eta, move, rmin);
    rho_new[e] = v;
    chg = fmax(chg, fabs(v - rho[e]));
  }
  __shared__ double sm[kTopThreads];
  sm[threadIdx.x] = chg;
  __syncthreads();
  for (int o = kTopThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
  if (last_cta(ticket)) {
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int i = 0; i < (int)gridDim.x; ++i) a = fmax(a, ((volatile double *)partials)[i]);
      st->change = a;
      st->lambda = lam;
    }
  }
}

cudaError_t launch_oc(const DeviceMesh &m, const double *rho, const double *dc, double eta, double move, double rmin,
                      double *rho_new, double *partials, unsigned int *ticket, OcState *st, int max_bisect,
                      cudaStream_t s) {
  const int g = top_grid(m.Ne);
  oc_init_kernel<<<g, kTopThreads, 0, s>>>(m.leaf, dc, m.Ne, m.L, m.h0, partials, ticket, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int i = 0; i < max_bisect; ++i) {
    oc_volume_kernel<<<g, kTopThreads, 0, s>>>(m.leaf, rho, dc, m.Ne, m.L, m.h0, eta, move, rmin, partials, ticket,
                                               st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  oc_final_kernel<<<g, kTopThreads, 0, s>>>(m.leaf, rho, dc, m.Ne, m.L, m.h0, eta, move, rmin, rho_new, partials,
                                            ticket, st);
  return cudaGetLastError();
}

}  // namespace amr
