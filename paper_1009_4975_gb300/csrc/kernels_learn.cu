// Transfers and optimiser of the learned initial guess (no paper counterpart; the network and
// its loss are defined with the C ABI in include/tm.h):
//   * network input on the uniform voxel grid of level g (X x Y x Z cells of side
//     hv = 2^(L-g) finest units): channel 0 the volume average of rho over each voxel, channels
//     1-3 the restriction P^T f of the loads divided by s = max |P^T f|;
//   * P: trilinear interpolation of cell-centred values at the mesh nodes, the cell index clamped
//     to [0, n-2] per axis so that the boundary half-cells extrapolate linearly (exact for
//     linear fields);
//   * the initial guess u0 = s P(out) on the A-space, and the gradient of the energy loss
//     0.5 u0^T A u0 - f^T u0 with respect to the network output, s P^T (A u0 - f);
//   * an Adam step on the parameters.
// Layouts: voxel arrays channel-major, z fastest (c, i, j, k); A-space vectors 3 per node.
// Restrictions are gathers over a node list grouped by each node's lower stencil cell, in a
// fixed order (no atomics).
#include <cuda_runtime.h>

#include "reduce.cuh"
#include "tm_internal.h"

namespace amr {

namespace {

constexpr int kT = 256;

int grid_of(int64_t n, int cap_per_sm = 8) {
  int64_t g = (n + kT - 1) / kT;
  if (g < 1) g = 1;
  if (g > cap_per_sm * device_sms()) g = cap_per_sm * device_sms();
  return (int)g;
}

// lower stencil cell and the weight of the upper one along one axis (finest-unit coordinate p)
__device__ __forceinline__ void axis_weight(int p, int n, int hv, int &i0, double &t) {
  const double u = (double)p / hv - 0.5;
  int i = (int)floor(u);
  i = i < 0 ? 0 : (i > n - 2 ? n - 2 : i);
  i0 = i;
  t = u - i;
}

__global__ void voxel_density_kernel(const int32_t *cellmap, const double *rho, int fx, int fy, int vs, int X, int Y,
                                     int Z, float *out) {
  const int64_t nv = (int64_t)X * Y * Z;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(v % Z), j = (int)((v / Z) % Y), i = (int)(v / ((int64_t)Y * Z));
    double s = 0.0;
    for (int c = 0; c < vs; ++c)
      for (int b = 0; b < vs; ++b)
        for (int a = 0; a < vs; ++a)
          s += rho[cellmap[((size_t)(k * vs + c) * fy + (j * vs + b)) * fx + (i * vs + a)]];
    out[v] = (float)(s / ((double)vs * vs * vs));
  }
}

// pf(c, i, j, k) = sum over nodes n of w_n(i, j, k) v[3 n + c], v = a - b (b may be NULL), as a
// gather over the nodes of the <= 8 stencil cells whose trilinear stencils include (i, j, k).
__global__ void voxel_restrict_kernel(const double *a, const double *b, const int32_t *vptr, const int32_t *vnode,
                                      const int32_t *nxyz, const uint8_t *nflag, int hv, int X, int Y, int Z,
                                      double *pf) {
  const int64_t nv = (int64_t)X * Y * Z;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(v % Z), j = (int)((v / Z) % Y), i = (int)(v / ((int64_t)Y * Z));
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int ai = i - 1; ai <= i; ++ai) {
      if (ai < 0 || ai > X - 2) continue;
      for (int aj = j - 1; aj <= j; ++aj) {
        if (aj < 0 || aj > Y - 2) continue;
        for (int ak = k - 1; ak <= k; ++ak) {
          if (ak < 0 || ak > Z - 2) continue;
          const int64_t anc = ((int64_t)ai * Y + aj) * Z + ak;
          for (int q = vptr[anc]; q < vptr[anc + 1]; ++q) {
            const int n = vnode[q];
            if (nflag[n]) continue;       // constrained nodes carry no A-space value
            int i0, j0, k0;
            double tx, ty, tz;
            axis_weight(nxyz[3 * n], X, hv, i0, tx);
            axis_weight(nxyz[3 * n + 1], Y, hv, j0, ty);
            axis_weight(nxyz[3 * n + 2], Z, hv, k0, tz);
            const double w = (i == i0 ? 1.0 - tx : tx) * (j == j0 ? 1.0 - ty : ty) * (k == k0 ? 1.0 - tz : tz);
            const double *va = a + 3 * (size_t)n;
            double v0 = va[0], v1 = va[1], v2 = va[2];
            if (b) {
              const double *vb = b + 3 * (size_t)n;
              v0 -= vb[0]; v1 -= vb[1]; v2 -= vb[2];
            }
            s0 += w * v0; s1 += w * v1; s2 += w * v2;
          }
        }
      }
    }
    pf[v] = s0;
    pf[nv + v] = s1;
    pf[2 * nv + v] = s2;
  }
}

// max |pf| over all entries (per-CTA partials, the last CTA finishes; max is order independent)
__global__ void __launch_bounds__(kT) absmax_kernel(const double *x, int64_t n, double *partials,
                                                    unsigned int *ticket, double *out) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  __shared__ double sm[kT];
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
  if (last_cta(ticket)) {
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kT) t = fmax(t, ((volatile double *)partials)[i]);
    sm[threadIdx.x] = t;
    __syncthreads();
    for (int o = kT / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
      __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
  }
}

// x[1 + c](i, j, k) = pf(c, i, j, k) / s, channels after the density; s from the device.
__global__ void scale_input_kernel(const double *pf, const double *s, int64_t nv, float *x) {
  const double inv = 1.0 / *s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * nv; i += (int64_t)gridDim.x * blockDim.x)
    x[nv + i] = (float)(pf[i] * inv);
}

// dout(c, i, j, k) = s * pf(c, i, j, k)
__global__ void scale_grad_kernel(const double *pf, double s, int64_t n, float *dout) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dout[i] = (float)(s * pf[i]);
}

// u0 = s P(out) at the free nodes, 0 at constrained ones
__global__ void voxel_prolong_kernel(const float *out, const int32_t *nxyz, const uint8_t *nflag, int64_t Nn, int hv,
                                     int X, int Y, int Z, double s, double *u0) {
  const int64_t nv = (int64_t)X * Y * Z;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < Nn; n += (int64_t)gridDim.x * blockDim.x) {
    double v[3] = {0.0, 0.0, 0.0};
    if (!nflag[n]) {
      int i0, j0, k0;
      double tx, ty, tz;
      axis_weight(nxyz[3 * n], X, hv, i0, tx);
      axis_weight(nxyz[3 * n + 1], Y, hv, j0, ty);
      axis_weight(nxyz[3 * n + 2], Z, hv, k0, tz);
      for (int q = 0; q < 8; ++q) {
        const int a = q & 1, b = (q >> 1) & 1, c = q >> 2;
        const double w = (a ? tx : 1.0 - tx) * (b ? ty : 1.0 - ty) * (c ? tz : 1.0 - tz);
        const int64_t cell = ((int64_t)(i0 + a) * Y + (j0 + b)) * Z + (k0 + c);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) v[ch] += w * (double)out[ch * nv + cell];
      }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) u0[3 * n + ch] = s * v[ch];
  }
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

cudaError_t learn_input_launch(const DeviceMesh &m, const LearnTables &t, const double *rho, const double *f,
                               double *pf, double *partials, unsigned int *ticket, double *s_dev, float *x,
                               cudaStream_t st) {
  const int64_t nv = (int64_t)t.X * t.Y * t.Z;
  voxel_density_kernel<<<grid_of(nv), kT, 0, st>>>(m.cellmap, rho, m.fx, m.fy, t.hv, t.X, t.Y, t.Z, x);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  voxel_restrict_kernel<<<grid_of(nv), kT, 0, st>>>(f, nullptr, t.vptr, t.vnode, t.nxyz, m.nflag, t.hv, t.X, t.Y, t.Z,
                                                     pf);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  absmax_kernel<<<grid_of(3 * nv, 4), kT, 0, st>>>(pf, 3 * nv, partials, ticket, s_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  scale_input_kernel<<<grid_of(3 * nv), kT, 0, st>>>(pf, s_dev, nv, x);
  return cudaGetLastError();
}

cudaError_t learn_guess_launch(const DeviceMesh &m, const LearnTables &t, const float *out, double s, double *u0,
                               cudaStream_t st) {
  voxel_prolong_kernel<<<grid_of(m.Nn), kT, 0, st>>>(out, t.nxyz, m.nflag, m.Nn, t.hv, t.X, t.Y, t.Z, s, u0);
  return cudaGetLastError();
}

cudaError_t learn_grad_launch(const DeviceMesh &m, const LearnTables &t, const double *au0, const double *f, double s,
                              double *pf, float *dout, cudaStream_t st) {
  const int64_t nv = (int64_t)t.X * t.Y * t.Z;
  voxel_restrict_kernel<<<grid_of(nv), kT, 0, st>>>(au0, f, t.vptr, t.vnode, t.nxyz, m.nflag, t.hv, t.X, t.Y, t.Z,
                                                     pf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scale_grad_kernel<<<grid_of(3 * nv), kT, 0, st>>>(pf, s, 3 * nv, dout);
  return cudaGetLastError();
}

cudaError_t adam_launch(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st) {
  adam_kernel<<<grid_of(n), kT, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace amr
