// Dynamic mesh adaptation on the device (paper Sec. 4): refinement/derefinement
// marks, the sibling sweep and the incompatibility sweep; the design difference of
// Eq. 10 on the finest grid; and the transfer of the displacement to the nodes of an
// adapted mesh (the warm start after remeshing).
//
// Marks: +1 refine, 0 keep, -1 derefine.
//  * mark: element e is solid when rho_e >= rho_s; it is marked +1 when it is
//    solid or the centre of some solid element lies at a distance below r_AMR from
//    its centre (compared exactly, see amr_mark_kernel), else -1.  Finest-level elements cannot refine and level-0 elements cannot
//    derefine (0).  Solid neighbours are found through the finest-cell map over
//    the box [c - r_AMR, c + r_AMR], stopping at the first one.
//  * sibling sweep: a -1 survives only when all 8 children of its parent are
//    leaves marked -1.
//  * incompatibility sweep: a -1 survives only when every leaf whose closure meets
//    the parent box ends at most one level finer than the parent, each such leaf
//    taken at its level after its own refinement (coarsenings of neighbours are
//    ignored: order independent).  All 8 siblings see the same parent box and so
//    decide alike.
#include <cuda_runtime.h>

#include "reduce.cuh"
#include "tm_internal.h"

namespace amr {

constexpr int kAmrThreads = 256;

__device__ __forceinline__ int cell_owner(const int32_t *cellmap, int fx, int fy, int x, int y, int z) {
  return cellmap[((size_t)z * fy + y) * fx + x];
}

// Distances are compared exactly: centres in half finest-cell units are integers
// (2 * anchor + size), so the squared distance d2 is an exact integer, and "distance
// below r_AMR" is d2 < thr with thr = (2 r_AMR / unit)^2 (computed once in FP64).
__global__ void __launch_bounds__(kAmrThreads) amr_mark_kernel(const int32_t *leaf, const int32_t *cellmap, int fx,
                                                               int fy, int fz, int L, double ru, double thr,
                                                               const double *rho, double rho_solid, int64_t Ne,
                                                               int8_t *mark) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    const int *le = leaf + 4 * e;
    const int se = 1 << (L - le[3]);
    bool refine = rho[e] >= rho_solid;
    if (!refine) {
      const int c2[3] = {2 * le[0] + se, 2 * le[1] + se, 2 * le[2] + se};
      const int ext[3] = {fx, fy, fz};
      int lo[3], hi[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        // cells that can hold the centre of an element closer than r_AMR, one cell of margin
        lo[a] = (int)floor(0.5 * c2[a] - ru) - 1;
        hi[a] = (int)ceil(0.5 * c2[a] + ru);
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > ext[a] - 1) hi[a] = ext[a] - 1;
      }
      for (int iz = lo[2]; iz <= hi[2] && !refine; ++iz)
        for (int iy = lo[1]; iy <= hi[1] && !refine; ++iy)
          for (int ix = lo[0]; ix <= hi[0] && !refine; ++ix) {
            const int d = cell_owner(cellmap, fx, fy, ix, iy, iz);
            if (!(rho[d] >= rho_solid)) continue;
            const int *ld = leaf + 4 * d;
            const int sd = 1 << (L - ld[3]);
            const long long dx = 2 * ld[0] + sd - c2[0], dy = 2 * ld[1] + sd - c2[1], dz = 2 * ld[2] + sd - c2[2];
            if ((double)(dx * dx + dy * dy + dz * dz) < thr) refine = true;
          }
    }
    int8_t m = refine ? 1 : -1;
    if (m == 1 && le[3] >= L) m = 0;
    if (m == -1 && le[3] == 0) m = 0;
    mark[e] = m;
  }
}

__global__ void __launch_bounds__(kAmrThreads) amr_sweep_siblings_kernel(const int32_t *leaf, const int32_t *cellmap,
                                                                         int fx, int fy, int L, const int8_t *in,
                                                                         int64_t Ne, int8_t *out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    int8_t m = in[e];
    if (m == -1) {
      const int *le = leaf + 4 * e;
      const int s = 1 << (L - le[3]);
      const int pa[3] = {le[0] / (2 * s) * (2 * s), le[1] / (2 * s) * (2 * s), le[2] / (2 * s) * (2 * s)};
      for (int k = 0; k < 8 && m == -1; ++k) {
        const int ax = pa[0] + s * (k & 1), ay = pa[1] + s * ((k >> 1) & 1), az = pa[2] + s * ((k >> 2) & 1);
        const int d = cell_owner(cellmap, fx, fy, ax, ay, az);
        const int *ld = leaf + 4 * d;
        if (ld[3] != le[3] || ld[0] != ax || ld[1] != ay || ld[2] != az || in[d] != -1) m = 0;
      }
    }
    out[e] = m;
  }
}

__global__ void __launch_bounds__(kAmrThreads) amr_sweep_balance_kernel(const int32_t *leaf, const int32_t *cellmap,
                                                                        int fx, int fy, int fz, int L,
                                                                        const int8_t *in, int64_t Ne, int8_t *out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < Ne; e += (int64_t)gridDim.x * blockDim.x) {
    int8_t m = in[e];
    if (m == -1) {
      const int *le = leaf + 4 * e;
      const int s = 1 << (L - le[3]);
      const int ps = 2 * s;
      const int pa[3] = {le[0] / ps * ps, le[1] / ps * ps, le[2] / ps * ps};
      const int lo[3] = {max(pa[0] - 1, 0), max(pa[1] - 1, 0), max(pa[2] - 1, 0)};
      const int hi[3] = {min(pa[0] + ps + 1, fx), min(pa[1] + ps + 1, fy), min(pa[2] + ps + 1, fz)};
      // only the one-cell shell around the parent box can hold other leaves
      for (int z = lo[2]; z < hi[2] && m == -1; ++z)
        for (int y = lo[1]; y < hi[1] && m == -1; ++y)
          for (int x = lo[0]; x < hi[0] && m == -1; ++x) {
            const bool inside = x >= pa[0] && x < pa[0] + ps && y >= pa[1] && y < pa[1] + ps && z >= pa[2] &&
                                z < pa[2] + ps;
            if (inside) continue;
            const int d = cell_owner(cellmap, fx, fy, x, y, z);
            const int nl = leaf[4 * d + 3] + (in[d] == 1 ? 1 : 0);
            if (nl > le[3]) m = 0;
          }
    }
    out[e] = m;
  }
}

int amr_grid(int64_t n) {
  int64_t g = (n + kAmrThreads - 1) / kAmrThreads;
  if (g < 1) g = 1;
  if (g > 8 * device_sms()) g = 8 * device_sms();
  return (int)g;
}

cudaError_t launch_amr_mark(const DeviceMesh &m, const double *rho, double rho_solid, double r_amr, int8_t *tmp,
                            int8_t *mark, cudaStream_t s) {
  const int g = amr_grid(m.Ne);
  const double t = 2.0 * r_amr / m.hmin;
  amr_mark_kernel<<<g, kAmrThreads, 0, s>>>(m.leaf, m.cellmap, m.fx, m.fy, m.fz, m.L, r_amr / m.hmin, t * t, rho,
                                            rho_solid, m.Ne, mark);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  amr_sweep_siblings_kernel<<<g, kAmrThreads, 0, s>>>(m.leaf, m.cellmap, m.fx, m.fy, m.L, mark, m.Ne, tmp);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  amr_sweep_balance_kernel<<<g, kAmrThreads, 0, s>>>(m.leaf, m.cellmap, m.fx, m.fy, m.fz, m.L, tmp, m.Ne, mark);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Eq. 10
__global__ void paint_kernel(const int32_t *leaves, int64_t n, int fx, int fy, int L, int32_t *map) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int *lf = leaves + 4 * i;
    const int s = 1 << (L - lf[3]);
    for (int z = 0; z < s; ++z)
      for (int y = 0; y < s; ++y)
        for (int x = 0; x < s; ++x)
          map[((size_t)(lf[2] + z) * fy + (lf[1] + y)) * fx + (lf[0] + x)] = (int32_t)i;
  }
}

// sums over finest cells of |rho1 - rho2| and rho1 (FP64, fixed order per CTA, last CTA finishes)
__global__ void __launch_bounds__(kAmrThreads) design_diff_kernel(const int32_t *map1, const double *rho1,
                                                                  const int32_t *map2, const double *rho2,
                                                                  int64_t ncell, double *partials,
                                                                  unsigned int *ticket, double *out) {
  double num = 0.0, den = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = map2[c];   // every cell is painted: the host checked the tiling
    const double a = rho1[map1[c]], b = rho2[j < 0 ? 0 : j];
    num += fabs(a - b);
    den += a;
  }
  block_sum2<kAmrThreads>(num, den);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = num;
    partials[2 * blockIdx.x + 1] = den;
  }
  if (last_cta(ticket)) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kAmrThreads) {
      s0 += ((volatile double *)partials)[2 * i];
      s1 += ((volatile double *)partials)[2 * i + 1];
    }
    block_sum2<kAmrThreads>(s0, s1);
    if (threadIdx.x == 0) {
      out[0] = s0;
      out[1] = s1;
    }
  }
}

cudaError_t launch_design_difference(const DeviceMesh &m, const double *rho1, const int32_t *leaves2, int64_t n2,
                                     const double *rho2, int32_t *map2, double *partials, unsigned int *ticket,
                                     double *out, cudaStream_t s) {
  paint_kernel<<<amr_grid(n2), kAmrThreads, 0, s>>>(leaves2, n2, m.fx, m.fy, m.L, map2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t ncell = (int64_t)m.fx * m.fy * m.fz;
  design_diff_kernel<<<amr_grid(ncell), kAmrThreads, 0, s>>>(m.cellmap, rho1, map2, rho2, ncell, partials, ticket,
                                                             out);
  return cudaGetLastError();
}

// Displacement transfer: the old mesh's finite-element field (u_full: hanging entries
// interpolated, so the field is continuous and trilinear on each leaf) evaluated at integer
// finest-grid points.  Each point takes the leaf covering a finest cell whose closed box holds it
// (coordinates clamped to the last cell), and the trilinear interpolation of that leaf's corner
// values.  Points outside the closed box are counted in *bad and give 0.
__global__ void __launch_bounds__(kAmrThreads) transfer_kernel(const int32_t *leaf, const int32_t *conn,
                                                               const int32_t *cellmap, int fx, int fy, int fz, int L,
                                                               const double *u_full, const int32_t *pts, int64_t n,
                                                               double *out, int *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
    if (px < 0 || py < 0 || pz < 0 || px > fx || py > fy || pz > fz) {
      atomicAdd(bad, 1);
      out[3 * i] = out[3 * i + 1] = out[3 * i + 2] = 0.0;
      continue;
    }
    const int e = cell_owner(cellmap, fx, fy, min(px, fx - 1), min(py, fy - 1), min(pz, fz - 1));
    const int *l = leaf + 4 * (size_t)e;
    const double s = (double)(1 << (L - l[3]));
    const double tx = (px - l[0]) / s, ty = (py - l[1]) / s, tz = (pz - l[2]) / s;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double w = ((k & 1) ? tx : 1.0 - tx) * (((k >> 1) & 1) ? ty : 1.0 - ty) * (((k >> 2) & 1) ? tz : 1.0 - tz);
      const double *uc = u_full + 3 * (size_t)conn[8 * (size_t)e + k];
      v0 += w * uc[0];
      v1 += w * uc[1];
      v2 += w * uc[2];
    }
    out[3 * i] = v0;
    out[3 * i + 1] = v1;
    out[3 * i + 2] = v2;
  }
}

cudaError_t launch_transfer(const DeviceMesh &m, const double *u_full, const int32_t *pts, int64_t n, double *out,
                            int *bad, cudaStream_t s) {
  int64_t g = (n + kAmrThreads - 1) / kAmrThreads;
  if (g < 1) g = 1;
  if (g > 8 * device_sms()) g = 8 * device_sms();
  transfer_kernel<<<(int)g, kAmrThreads, 0, s>>>(m.leaf, m.conn, m.cellmap, m.fx, m.fy, m.fz, m.L, u_full, pts, n, out,
                                                  bad);
  return cudaGetLastError();
}

}  // namespace amr
