// Optimisation-step kernels: compliance sensitivities (paper Sec. 3), the
// filters of Eq. 3-5, and the optimality-criteria update with a device-side
// bracket search for the Lagrange multiplier of the volume constraint.
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
    double rp1, rp;   // rho^(p-1) and rho^p: exact products for the common integer penalties
    if (penal == 3.0) { rp1 = r * r; rp = rp1 * r; }
    else if (penal == 1.0) { rp1 = 1.0; rp = r; }
    else if (penal == 2.0) { rp1 = r; rp = r * r; }
    else { rp1 = pow(r, penal - 1.0); rp = pow(r, penal); }
    dc[e] = -penal * rp1 * (E0 - Emin) * h * en;
    cpart += (Emin + rp * (E0 - Emin)) * h * en;
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
// order (the componentwise max of its anchor and the box's low corner); along x
// the scan jumps past the rest of each leaf's cells.  Centre offsets are whole
// numbers of half finest cells, so the squared distance D2 in those units is an
// exact integer, below (2 rmin / h_min)^2 <= 64 for a neighbour; the weight
// H_de V_d = (rmin - dist) h_d^3 then depends only on (level of d, D2) and comes
// from a per-block table, with dist = sqrt(D2) h_min / 2.
constexpr int kFilterD2 = 65;        // D2 in [0, 64]
constexpr int kFilterLevels = 13;    // max_level <= 12
__global__ void __launch_bounds__(kTopThreads) filter_kernel(const int4 *leaf, const int32_t *cellmap, int fx,
                                                             int fy, int fz, int L, double unit, const double *rho,
                                                             const double *x, double rmin, int mode, int64_t Ne,
                                                             double *out) {
  __shared__ double W[kFilterLevels * kFilterD2];
  for (int i = threadIdx.x; i < (L + 1) * kFilterD2; i += blockDim.x) {
    const int lev = i / kFilterD2, D2 = i % kFilterD2;
    const double dist = sqrt((double)D2) * (0.5 * unit);
    const double hd = ldexp(unit, L - lev);
    W[i] = dist < rmin ? (rmin - dist) * hd * hd * hd : 0.0;
  }
  __syncthreads();
  const double ru = rmin / unit;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    const int4 le = leaf[e];
    const int se = 1 << (L - le.w);
    // centre in half finest cells
    const int c2[3] = {2 * le.x + se, 2 * le.y + se, 2 * le.z + se};
    const int ext[3] = {fx, fy, fz};
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // cells i with i < c + ru and i + 1 > c - ru (c = c2 / 2, exact)
      const double c = 0.5 * c2[a];
      lo[a] = (int)floor(c - ru);
      hi[a] = (int)ceil(c + ru) - 1;
      if (lo[a] < 0) lo[a] = 0;
      if (hi[a] > ext[a] - 1) hi[a] = ext[a] - 1;
    }
    double num = 0.0, den = 0.0;
    for (int iz = lo[2]; iz <= hi[2]; ++iz)
      for (int iy = lo[1]; iy <= hi[1]; ++iy)
        for (int ix = lo[0]; ix <= hi[0];) {
          const int d = cellmap[((size_t)iz * fy + iy) * fx + ix];
          const int4 ld = leaf[d];
          const int sd = 1 << (L - ld.w);
          ix = ld.x + sd;   // the next leaf along x; this one is first seen at max(ld.x, lo[0])
          if (iy != (ld.y > lo[1] ? ld.y : lo[1]) || iz != (ld.z > lo[2] ? ld.z : lo[2])) continue;
          const int dx = abs(2 * ld.x + sd - c2[0]), dy = abs(2 * ld.y + sd - c2[1]), dz = abs(2 * ld.z + sd - c2[2]);
          if (dx > 8 || dy > 8 || dz > 8) continue;
          const int D2 = dx * dx + dy * dy + dz * dz;
          if (D2 >= kFilterD2) continue;
          const double w = W[ld.w * kFilterD2 + D2];
          if (w == 0.0) continue;
          num += mode == 0 ? w * rho[d] * x[d] : w * x[d];
          den += w;
        }
    out[e] = mode == 0 ? num / (rho[e] * den) : num / den;
  }
}

cudaError_t launch_filter(const DeviceMesh &m, const double *rho, const double *x, double rmin, int mode,
                          double *out, cudaStream_t s) {
  filter_kernel<<<top_grid(m.Ne), kTopThreads, 0, s>>>(reinterpret_cast<const int4 *>(m.leaf), m.cellmap, m.fx, m.fy, m.fz, m.L, m.hmin, rho, x, rmin,
                                                       mode, m.Ne, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- OC
// rho_new = clamp(rho (g / (lambda V))^eta, lo, hi) with g = max(-dc, 0), lo = max(rho_min, rho - move),
// hi = min(1, rho + move).  With s = lambda^-eta and the lambda-free factor a_e = rho_e (g_e / V_e)^eta,
// rho_new_e = clamp(a_e s, lo_e, hi_e) and the volume
//   vol(s) = sum_e V_e clamp(a_e s, lo_e, hi_e)
// is a non-decreasing, piecewise linear function of s whose slope at s is the sum of a_e V_e over
// the elements strictly between their bounds.  oc_init_kernel tabulates (a_e, lo_e, hi_e, V_e) once
// per update; each oc_search_kernel launch evaluates vol (and the slope) at one or two candidates
// from OcState in FP64 and, in its last CTA, narrows the bracket [s_lo, s_hi] around the root of
// vol(s) = target and picks the next candidates: a Newton step on the piecewise linear volume when
// it stays inside the bracket and, once the bracket is bounded, shrinks (to below half the previous
// step), else a bisection of
// the bracket (geometric while s_hi > 2 s_lo, by 16x while s_hi is unbounded).  Once a Newton step
// is below 1e-4 relative, the next launch evaluates the pair s (1 -+ 0.4 tol eta), which closes the
// bracket if the step was accurate.  The search stops when the bracket's relative width in lambda
// is below tol (s_hi - s_lo <= tol eta (s_lo + s_hi)) or a candidate hits the target exactly;
// lambda is then the midpoint of the lambda bracket.  Launches after that return at once.  The
// initial bracket is the bisection's: lambda in (0, 1e9 max g / min V].
__global__ void __launch_bounds__(kTopThreads) oc_init_kernel(const int32_t *leaf, const double *rho,
                                                              const double *dc, int64_t Ne, int L, double h0,
                                                              double eta, double move, double rmin,
                                                              double4_32a *tab, double *partials,
                                                              unsigned int *ticket, OcState *st) {
  double gmax = 0.0, vmin = 1e300, asum = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    const double g = fmax(-dc[e], 0.0);
    const double h = ldexp(h0, -leaf[4 * e + 3]);
    const double V = h * h * h;
    const double r = rho[e];
    const double t = g / V;
    const double ae = r * (eta == 0.5 ? sqrt(t) : pow(t, eta));
    tab[e] = make_double4_32a(ae, fmax(rmin, r - move), fmin(1.0, r + move), V);
    gmax = fmax(gmax, g);
    vmin = fmin(vmin, V);
    asum += ae * V;
  }
  asum = block_sum<kTopThreads>(asum);
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
    partials[blockIdx.x] = sm[0];
    partials[gridDim.x + blockIdx.x] = sv[0];
    partials[2 * gridDim.x + blockIdx.x] = asum;
  }
  if (last_cta(ticket)) {
    const double A = sum_partials<kTopThreads>(partials + 2 * gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      double a = 0.0, b = 1e300;
      for (int i = 0; i < (int)gridDim.x; ++i) {
        a = fmax(a, ((volatile double *)partials)[i]);
        b = fmin(b, ((volatile double *)partials)[gridDim.x + i]);
      }
      const double lmax = 1e9 * fmax(a, 1e-300) / b;
      st->s_lo = eta == 0.5 ? 1.0 / sqrt(lmax) : pow(lmax, -eta);
      st->s_hi = INFINITY;
      // first candidate: the root if no element were clamped
      double c = A > 0.0 ? st->target / A : 0.0;
      if (!(c > st->s_lo) || !isfinite(c)) c = 16.0 * st->s_lo;
      st->c0 = c;
      st->c1 = -1.0;
      st->step = INFINITY;
      st->done = 0;
      st->iters = 0;
    }
  }
}

// lambda^-eta (the exact square root for the default eta = 1/2) and its inverse
__device__ __forceinline__ double lam_factor(double lam, double eta) {
  return eta == 0.5 ? 1.0 / sqrt(lam) : pow(lam, -eta);
}
__device__ __forceinline__ double lam_of(double sfac, double eta) {
  return eta == 0.5 ? 1.0 / (sfac * sfac) : pow(sfac, -1.0 / eta);
}

__global__ void __launch_bounds__(kTopThreads) oc_search_kernel(const double4_32a *tab, int64_t Ne, double eta,
                                                                double *partials, unsigned int *ticket,
                                                                OcState *st) {
  if (st->done) return;
  const double c0 = st->c0, c1 = st->c1;
  double v0 = 0.0, a0 = 0.0, v1 = 0.0;
  if (c1 > 0.0) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
      const double4_32a t = tab[e];
      const double x0 = t.x * c0;
      v0 += fmin(fmax(x0, t.y), t.z) * t.w;
      if (x0 > t.y && x0 < t.z) a0 += t.x * t.w;
      v1 += fmin(fmax(t.x * c1, t.y), t.z) * t.w;
    }
  } else {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
      const double4_32a t = tab[e];
      const double x0 = t.x * c0;
      v0 += fmin(fmax(x0, t.y), t.z) * t.w;
      if (x0 > t.y && x0 < t.z) a0 += t.x * t.w;
    }
  }
  block_sum2<kTopThreads>(v0, a0);
  v1 = block_sum<kTopThreads>(v1);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v0;
    partials[gridDim.x + blockIdx.x] = a0;
    partials[2 * gridDim.x + blockIdx.x] = v1;
  }
  if (!last_cta(ticket)) return;
  const double V0 = sum_partials<kTopThreads>(partials, gridDim.x);
  const double A0 = sum_partials<kTopThreads>(partials + gridDim.x, gridDim.x);
  const double V1 = sum_partials<kTopThreads>(partials + 2 * gridDim.x, gridDim.x);
  if (threadIdx.x != 0) return;
  const double T = st->target;
  double lo = st->s_lo, hi = st->s_hi;
  bool exact = false;
  double root = 0.0;
  // vol is non-decreasing: vol(c) > T puts the root below c, vol(c) < T above it
  if (V0 > T) hi = fmin(hi, c0);
  else if (V0 < T) lo = fmax(lo, c0);
  else { exact = true; root = c0; }
  if (c1 > 0.0 && !exact) {
    if (V1 > T) hi = fmin(hi, c1);
    else if (V1 < T) lo = fmax(lo, c1);
    else { exact = true; root = c1; }
  }
  st->s_lo = lo;
  st->s_hi = hi;
  st->iters += 1;
  const double tol_s = st->tol * eta;
  if (exact || (hi < INFINITY && hi - lo <= tol_s * (lo + hi))) {
    st->l1 = exact ? lam_of(root, eta) : lam_of(hi, eta);
    st->l2 = exact ? st->l1 : lam_of(lo, eta);
    st->lambda = 0.5 * (st->l1 + st->l2);
    st->done = 1;
    return;
  }
  double next = -1.0;
  if (A0 > 0.0) {
    const double sn = c0 + (T - V0) / A0;
    const double step = fabs(sn - c0);
    if (isfinite(sn) && sn > lo && sn < hi && (step < 0.5 * st->step || hi == INFINITY)) {
      st->step = step;
      if (step <= 1e-4 * sn) {
        const double d = 0.4 * tol_s * sn;
        const double p0 = sn - d, p1 = sn + d;
        if (p0 > lo && p1 < hi) {
          st->c0 = p0;
          st->c1 = p1;
          return;
        }
      }
      next = sn;
    }
  }
  if (next < 0.0) {
    next = hi == INFINITY ? 16.0 * lo : (hi > 2.0 * lo ? sqrt(lo) * sqrt(hi) : 0.5 * (lo + hi));
    st->step = INFINITY;
  }
  st->c0 = next;
  st->c1 = -1.0;
}

__global__ void __launch_bounds__(kTopThreads) oc_final_kernel(const double4_32a *tab, const double *rho, int64_t Ne,
                                                               double eta, double *rho_new, double *partials,
                                                               unsigned int *ticket, OcState *st) {
  // if the step limit ran out, lambda is the midpoint of the bracket reached
  const double lam = st->done ? st->lambda
                              : 0.5 * (lam_of(st->s_lo, eta) + (st->s_hi < INFINITY ? lam_of(st->s_hi, eta) : 0.0));
  const double sc = lam_factor(lam, eta);
  double chg = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    const double4_32a t = tab[e];
    const double v = fmin(fmax(t.x * sc, t.y), t.z);
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

cudaError_t launch_oc_init(const DeviceMesh &m, const double *rho, const double *dc, double eta, double move,
                           double rmin, double4_32a *tab, double *partials, unsigned int *ticket, OcState *st,
                           cudaStream_t s) {
  oc_init_kernel<<<top_grid(m.Ne), kTopThreads, 0, s>>>(m.leaf, rho, dc, m.Ne, m.L, m.h0, eta, move, rmin, tab,
                                                        partials, ticket, st);
  return cudaGetLastError();
}

cudaError_t launch_oc_search(const DeviceMesh &m, double eta, const double4_32a *tab, double *partials,
                             unsigned int *ticket, OcState *st, int steps, cudaStream_t s) {
  const int g = top_grid(m.Ne);
  for (int i = 0; i < steps; ++i) {
    oc_search_kernel<<<g, kTopThreads, 0, s>>>(tab, m.Ne, eta, partials, ticket, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_oc_final(const DeviceMesh &m, const double *rho, double eta, const double4_32a *tab,
                            double *rho_new, double *partials, unsigned int *ticket, OcState *st, cudaStream_t s) {
  oc_final_kernel<<<top_grid(m.Ne), kTopThreads, 0, s>>>(tab, rho, m.Ne, eta, rho_new, partials, ticket, st);
  return cudaGetLastError();
}

}  // namespace amr
