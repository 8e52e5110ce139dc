// Two-level preconditioner of the mixed solver: a Galerkin coarse correction on the vertex
// lattice of the base grid, approximated by a V-cycle over halved uniform lattices.  The
// paper's solver carries the slow part of the spectrum from solve to solve with a recycled
// Krylov subspace (Sec. 5); this coarse space takes that role here (no paper counterpart).
//
//   M^-1 r = D^-1 r + P0 V_0(P0^T r)
//
// * P0: trilinear interpolation of lattice values at the free mesh nodes.  Every leaf lies in
//   one base cell, so each lattice function is trilinear on each leaf and agrees with the
//   hanging-node interpolation (Eq. 6): the coarse space is nested in the finite-element space.
// * Level operators.  With nesting, P0^T A P0 is the stiffness of the lattice's trilinear cell
//   basis with the mesh's piecewise-constant Young's modulus.  Per cell C it is
//       K_C = (2/H)^2 sum_abc Q_abc mu_abc(C),   mu_abc(C) = int_C E(x) s_x^a s_y^b s_z^c dx,
//   with s in [-1, 1]^3 the cell's centred coordinates and Q_abc fixed 24 x 24 matrices (the
//   D-weighted products of the basis gradients, tabulated on the host).  The 27 moments of a
//   base cell are exact sums over its leaves (products of 1D integrals); a parent cell's
//   moments are exact affine transforms of its 8 children's, which gives the Galerkin
//   operator of every coarser level without forming P^T A P.
// * Cycle: l1-Jacobi sweeps (d_i = sum_j |A_ij| of the assembled level matrix), residual,
//   nodal restriction, recursion, prolongation, the same sweeps; the coarsest level is solved
//   by its dense inverse (formed on the host in FP64 from the FP64 cell matrices).
//
// Layout: level l has X x Y x Z cells and (X+1)(Y+1)(Z+1) nodes, node I = i + (X+1)(j + (Y+1)k),
// DOF 3 I + c; DOFs of nodes on clamped faces are kept at 0.  Cell matrices: [cell][24][24],
// local DOF 3 q + c of corner q = a + 2b + 4c.  All summation orders are fixed (no atomics).
// Several load cases run through one launch: grid dimension y (x for the coarsest solve) is the
// case, each case with its own level vectors (consecutive, one level's length apart), its own
// CG scalars and its own done flag; cases whose run is done return at once.
#include <cuda_runtime.h>

#include <utility>

#include "pcg.cuh"
#include "pdl.cuh"
#include "reduce.cuh"
#include "tm_internal.h"

namespace amr {

namespace {

constexpr int kT = 256;

// The load cases of a launch: case c0 + (grid index); sc (may be NULL) holds every case's CG
// scalars, and a case whose run is done is skipped.
struct Cases {
  const SolveScalars *sc;
  int c0;
};
__device__ __forceinline__ int case_of(const Cases &cs, int g) { return cs.c0 + g; }
__device__ __forceinline__ bool case_done(const Cases &cs, int c) {
  return cs.sc && *(volatile const int *)&cs.sc[c].done;
}
__device__ __forceinline__ int64_t lattice_len(int X, int Y, int Z) { return 3 * (int64_t)(X + 1) * (Y + 1) * (Z + 1); }

__device__ __forceinline__ bool lattice_fixed(int i, int j, int k, int X, int Y, int Z, unsigned faces) {
  return ((faces & 1u) && i == 0) || ((faces & 2u) && i == X) || ((faces & 4u) && j == 0) ||
         ((faces & 8u) && j == Y) || ((faces & 16u) && k == 0) || ((faces & 32u) && k == Z);
}

__device__ __forceinline__ double young(double r, double E0, double Emin, double p) {
  double rp;
  if (p == 3.0) rp = r * r * r;
  else if (p == 1.0) rp = r;
  else if (p == 2.0) rp = r * r;
  else rp = pow(r, p);
  return Emin + rp * (E0 - Emin);
}

// ---------------------------------------------------------------- set-up
// Moments of each base cell: one warp per cell over its leaves (a contiguous Morton range).
__global__ void moments0_kernel(const int32_t *cell_elem, const int32_t *leaf, const double *rho, int ncell, int X,
                                int Y, int L, double H, double E0, double Emin, double penal, double *mom) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= ncell) return;
  const int cx = warp % X, cy = (warp / X) % Y, cz = warp / (X * Y);
  const int S = 1 << L;
  const double invS = 1.0 / S;   // a power of two: dividing by S and multiplying by invS agree exactly
  const int o[3] = {cx * S, cy * S, cz * S};
  double m[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) m[q] = 0.0;
  const int e1 = cell_elem[2 * warp + 1];
  for (int e = cell_elem[2 * warp] + lane; e < e1; e += 32) {
    const int32_t *l = leaf + 4 * (int64_t)e;
    const int s = 1 << (L - l[3]);
    const double E = young(rho[e], E0, Emin, penal);
    double I[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double lo = 2.0 * (double)(l[a] - o[a]) * invS - 1.0, hi = 2.0 * (double)(l[a] + s - o[a]) * invS - 1.0;
      I[a][0] = 0.5 * H * (hi - lo);
      I[a][1] = 0.5 * H * (hi * hi - lo * lo) * 0.5;
      I[a][2] = 0.5 * H * (hi * hi * hi - lo * lo * lo) / 3.0;
    }
    double EI[9];   // ((E I_x) I_y), the leading products of the moment terms below
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) EI[a + 3 * b] = E * I[0][a] * I[1][b];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) m[a + 3 * b + 9 * c] += EI[a + 3 * b] * I[2][c];
  }
#pragma unroll
  for (int q = 0; q < 27; ++q) m[q] = warp_sum(m[q]);
  if (lane == 0)
    for (int q = 0; q < 27; ++q) mom[27 * (int64_t)warp + q] = m[q];
}

// Parent moments from the <= 8 children (the finer level has Xc x Yc x Zc cells, X = ceil(Xc / 2);
// children beyond the finer level's extent lie outside the box and carry nothing): per axis, a
// child with offset o (-1 lower, +1 upper) has s_parent = (s_child + o) / 2, so
//   m0' = m0,  m1' = (m1 + o m0) / 2,  m2' = (m2 + 2 o m1 + m0) / 4.
__global__ void moments_up_kernel(const double *mc, int Xc, int Yc, int Zc, int X, int Y, int Z, double *mp) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= X * Y * Z) return;
  const int px = p % X, py = (p / X) % Y, pz = p / (X * Y);
  double acc[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) acc[q] = 0.0;
  for (int ch = 0; ch < 8; ++ch) {
    const int ox = ch & 1, oy = (ch >> 1) & 1, oz = ch >> 2;
    if (2 * px + ox >= Xc || 2 * py + oy >= Yc || 2 * pz + oz >= Zc) continue;
    const int c = (2 * px + ox) + Xc * ((2 * py + oy) + Yc * (2 * pz + oz));
    double t[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) t[q] = mc[27 * (int64_t)c + q];
    const double sg[3] = {ox ? 1.0 : -1.0, oy ? 1.0 : -1.0, oz ? 1.0 : -1.0};
    // axis 0 (index a of t[a + 3b + 9c]), then 1, then 2
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int st = ax == 0 ? 1 : (ax == 1 ? 3 : 9);
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        const int base = ax == 0 ? 3 * r : (ax == 1 ? (r % 3) + 9 * (r / 3) : r);
        const double m0 = t[base], m1 = t[base + st], m2 = t[base + 2 * st];
        t[base + st] = 0.5 * (m1 + sg[ax] * m0);
        t[base + 2 * st] = 0.25 * (m2 + 2.0 * sg[ax] * m1 + m0);
      }
    }
#pragma unroll
    for (int q = 0; q < 27; ++q) acc[q] += t[q];
  }
#pragma unroll
  for (int q = 0; q < 27; ++q) mp[27 * (int64_t)p + q] = acc[q];
}

// K_C = (2/H)^2 sum_q Q_q mom_q, one thread per (cell, upper-triangle entry); FP64 accumulation
// over the moments whose coefficient is nonzero (in ascending q: the same sum as over all 27),
// stored to the entry and its mirror (the Q_q are symmetric).
__global__ void cellmat_kernel(const double *mom, const int32_t *qent, const uint8_t *qidx, const double *qval,
                               int ncell, double H, float *K32, double *K64) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)ncell * kCellUpper) return;
  const int64_t c = t / kCellUpper;
  const int u = (int)(t % kCellUpper);
  const int e = qent[u], i = e & 31, j = (e >> 5) & 31, nnz = e >> 10;
  const double *mc = mom + 27 * c;
  double s = 0.0;
  for (int k = 0; k < nnz; ++k) s += qval[u * kCellNnz + k] * mc[qidx[u * kCellNnz + k]];
  s *= 4.0 / (H * H);
  const int64_t a = 576 * c + 24 * i + j, b = 576 * c + 24 * j + i;
  if (K32) {
    K32[a] = (float)s;
    K32[b] = (float)s;
  }
  if (K64) {
    K64[a] = s;
    K64[b] = s;
  }
}

// Inverse l1 row sums of the assembled level matrix: d_(I,c) = sum over free neighbours J, c'
// of |sum over the cells holding I and J of K_C[(I,c),(J,c')]|.  0 at clamped nodes.
__global__ void l1diag_kernel(const float *K, int X, int Y, int Z, unsigned faces, float *dinv) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int nodes = (X + 1) * (Y + 1) * (Z + 1);
  if (I >= nodes) return;
  const int i = I % (X + 1), j = (I / (X + 1)) % (Y + 1), k = I / ((X + 1) * (Y + 1));
  if (lattice_fixed(i, j, k, X, Y, Z, faces)) {
    dinv[3 * I] = dinv[3 * I + 1] = dinv[3 * I + 2] = 0.f;
    return;
  }
  double s[3] = {0.0, 0.0, 0.0};
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int jx = i + dx, jy = j + dy, jz = k + dz;
        if (jx < 0 || jy < 0 || jz < 0 || jx > X || jy > Y || jz > Z) continue;
        if (lattice_fixed(jx, jy, jz, X, Y, Z, faces)) continue;
        double blk[3][3] = {};
        // cells holding both: per axis {i-1, i} for d = 0, {i-1} for d = -1, {i} for d = +1
        for (int cz = k - 1; cz <= k; ++cz) {
          if (cz < 0 || cz >= Z || cz > jz || cz + 1 < jz) continue;
          for (int cy = j - 1; cy <= j; ++cy) {
            if (cy < 0 || cy >= Y || cy > jy || cy + 1 < jy) continue;
            for (int cx = i - 1; cx <= i; ++cx) {
              if (cx < 0 || cx >= X || cx > jx || cx + 1 < jx) continue;
              const float *Kc = K + 576 * (int64_t)(cx + X * (cy + Y * cz));
              const int qi = (i - cx) + 2 * (j - cy) + 4 * (k - cz);
              const int qj = (jx - cx) + 2 * (jy - cy) + 4 * (jz - cz);
#pragma unroll
              for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int c2 = 0; c2 < 3; ++c2) blk[c][c2] += (double)Kc[(3 * qi + c) * 24 + 3 * qj + c2];
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) s[c] += fabs(blk[c][0]) + fabs(blk[c][1]) + fabs(blk[c][2]);
      }
#pragma unroll
  for (int c = 0; c < 3; ++c) dinv[3 * I + c] = s[c] > 0.0 ? (float)(1.0 / s[c]) : 0.f;
}

// ---------------------------------------------------------------- cycle
// Row (3 qi + c) of cell (cx, cy, cz) times the cell's x values: the part of (A x) at DOF (I, c)
// that the cell contributes, qi being node I's corner in the cell; x is 0 at clamped nodes.
__device__ __forceinline__ float cell_row_part(const float *K, const float *x, int cx, int cy, int cz, int qi, int c,
                                               int X, int Y) {
  const float4 *row = reinterpret_cast<const float4 *>(K + 576 * (int64_t)(cx + X * (cy + Y * cz)) + 24 * (3 * qi + c));
  float v[24];
#pragma unroll
  for (int w = 0; w < 6; ++w) {
    const float4 r4 = __ldg(row + w);
    v[4 * w] = r4.x; v[4 * w + 1] = r4.y; v[4 * w + 2] = r4.z; v[4 * w + 3] = r4.w;
  }
  float acc = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int J = (cx + (q & 1)) + (X + 1) * ((cy + ((q >> 1) & 1)) + (Y + 1) * (cz + (q >> 2)));
    acc = fmaf(v[3 * q], x[3 * J], acc);
    acc = fmaf(v[3 * q + 1], x[3 * J + 1], acc);
    acc = fmaf(v[3 * q + 2], x[3 * J + 2], acc);
  }
  return acc;
}

// mode 0: out = b - A x (residual).  mode 1: out = x + dinv (b - A x) (an l1-Jacobi sweep).
// mode 2: out = A x (b unused).  Eight threads per DOF, one per cell around its node (slot q:
// cell (i - 1 + q_x, j - 1 + q_y, k - 1 + q_z)), summed by a fixed shuffle tree over the eight, so
// that the small levels still spread over many SMs and every thread has one cell row to load.
__global__ void __launch_bounds__(kT) level_apply_kernel(const float *K, const float *x, const float *b,
                                                         const float *dinv, float *out, int X, int Y, int Z,
                                                         unsigned faces, int mode, Cases cs) {
  pdl_begin();
  const int cc = case_of(cs, blockIdx.y);
  if (case_done(cs, cc)) return;
  const int64_t off = cc * lattice_len(X, Y, Z);
  x += off;
  out += off;
  if (b) b += off;
  const int nodes = (X + 1) * (Y + 1) * (Z + 1);
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int t = (int)(g >> 3), q = (int)(g & 7);
  const bool live = t < 3 * nodes;
  bool fixed = true;
  float part = 0.f;
  if (live) {
    const int I = t / 3, c = t % 3;
    const int i = I % (X + 1), j = (I / (X + 1)) % (Y + 1), k = I / ((X + 1) * (Y + 1));
    fixed = lattice_fixed(i, j, k, X, Y, Z, faces);
    const int cx = i - 1 + (q & 1), cy = j - 1 + ((q >> 1) & 1), cz = k - 1 + (q >> 2);
    if (!fixed && cx >= 0 && cx < X && cy >= 0 && cy < Y && cz >= 0 && cz < Z)
      part = cell_row_part(K, x, cx, cy, cz, (i - cx) + 2 * (j - cy) + 4 * (k - cz), c, X, Y);
  }
  part += __shfl_xor_sync(0xffffffffu, part, 1);
  part += __shfl_xor_sync(0xffffffffu, part, 2);
  part += __shfl_xor_sync(0xffffffffu, part, 4);
  if (!live || q != 0) return;
  if (fixed) {
    out[t] = 0.f;
    return;
  }
  if (mode == 2) {
    out[t] = part;
    return;
  }
  const float r = b[t] - part;
  out[t] = mode == 0 ? r : fmaf(dinv[t], r, x[t]);
}

// Restriction of a level-l vector (Xf x Yf x Zf cells) to level l+1 (X, Y, Z cells): the
// transpose of nodal interpolation, weights 1 / 0.5 per axis.  With dinv: also x = dinv b
// (the first l1-Jacobi sweep from zero).
__global__ void __launch_bounds__(kT) level_restrict_kernel(const float *t_f, int Xf, int Yf, int Zf, int X, int Y,
                                                            int Z, unsigned faces, float *b_c, const float *dinv_c,
                                                            float *x_c, Cases cs) {
  pdl_begin();
  const int cc = case_of(cs, blockIdx.y);
  if (case_done(cs, cc)) return;
  t_f += cc * lattice_len(Xf, Yf, Zf);
  b_c += cc * lattice_len(X, Y, Z);
  if (x_c) x_c += cc * lattice_len(X, Y, Z);
  const int nodes = (X + 1) * (Y + 1) * (Z + 1);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nodes) return;
  const int J = t / 3, c = t % 3;
  const int i = J % (X + 1), j = (J / (X + 1)) % (Y + 1), k = J / ((X + 1) * (Y + 1));
  float s = 0.f;
  if (!lattice_fixed(i, j, k, X, Y, Z, faces)) {
    for (int dz = -1; dz <= 1; ++dz) {
      const int fz = 2 * k + dz;
      if (fz < 0 || fz > Zf) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int fy = 2 * j + dy;
        if (fy < 0 || fy > Yf) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int fx = 2 * i + dx;
          if (fx < 0 || fx > Xf) continue;
          const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f) * (dz ? 0.5f : 1.f);
          s = fmaf(w, t_f[3 * (fx + (Xf + 1) * (fy + (Yf + 1) * fz)) + c], s);
        }
      }
    }
  }
  b_c[t] = s;
  if (x_c) x_c[t] = dinv_c[t] * s;
}

// x_f += P x_c (X, Y, Z: the fine level's cells; Xc, Yc: the coarse level's): nodal
// interpolation from the halved lattice.
__global__ void __launch_bounds__(kT) level_prolong_kernel(const float *x_c, int Xc, int Yc, int Zc, int X, int Y,
                                                           int Z, unsigned faces, float *x_f, Cases cs) {
  pdl_begin();
  const int cc = case_of(cs, blockIdx.y);
  if (case_done(cs, cc)) return;
  x_c += cc * lattice_len(Xc, Yc, Zc);
  x_f += cc * lattice_len(X, Y, Z);
  const int nodes = (X + 1) * (Y + 1) * (Z + 1);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nodes) return;
  const int I = t / 3, c = t % 3;
  const int i = I % (X + 1), j = (I / (X + 1)) % (Y + 1), k = I / ((X + 1) * (Y + 1));
  if (lattice_fixed(i, j, k, X, Y, Z, faces)) return;
  float s = 0.f;
  for (int bz = 0; bz <= (k & 1); ++bz)
    for (int by = 0; by <= (j & 1); ++by)
      for (int bx = 0; bx <= (i & 1); ++bx) {
        const float w = ((i & 1) ? 0.5f : 1.f) * ((j & 1) ? 0.5f : 1.f) * ((k & 1) ? 0.5f : 1.f);
        const int J = (i / 2 + bx) + (Xc + 1) * ((j / 2 + by) + (Yc + 1) * (k / 2 + bz));
        s = fmaf(w, x_c[3 * J + c], s);
      }
  x_f[t] += s;
}

// Coarsest level: x = Ainv b over all of its DOFs (Ainv symmetric, zero rows and columns at
// clamped DOFs).  kDenseRows rows per CTA (grid x) and one CTA row per load case (grid y); one
// warp per row (lanes stride the row, then a fixed shuffle tree).
constexpr int kDenseRows = 8;
__global__ void __launch_bounds__(32 * kDenseRows) dense_solve_kernel(const float *Ainv, const float *b, float *x,
                                                                      int n, Cases cs) {
  pdl_begin();
  const int cc = case_of(cs, blockIdx.y);
  if (case_done(cs, cc)) return;
  b += (int64_t)cc * n;
  x += (int64_t)cc * n;
  extern __shared__ float sb[];
  for (int i = threadIdx.x; i < n; i += blockDim.x) sb[i] = b[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    const int r = blockIdx.x * kDenseRows + warp;
    if (r >= n) return;
    const float *row = Ainv + (int64_t)r * n;
    float s = 0.f;
    for (int j = lane; j < n; j += 32) s = fmaf(row[j], sb[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[r] = s;
  }
}

// ---------------------------------------------------------------- fine level <-> level 0
// Node code: bits 0-9, 10-19, 20-29: the node's position in its base cell in finest units
// (0 .. 2^L); bit 31: the node carries no unknowns (hanging or clamped).
__device__ __forceinline__ void trilinear8(uint32_t code, int L, float w[8]) {
  const float inv = 1.f / (float)(1 << L);
  const float tx = (float)(code & 1023u) * inv, ty = (float)((code >> 10) & 1023u) * inv,
              tz = (float)((code >> 20) & 1023u) * inv;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    w[q] = ((q & 1) ? tx : 1.f - tx) * ((q & 2) ? ty : 1.f - ty) * ((q & 4) ? tz : 1.f - tz);
}

// Stage 1 of P0^T r: one warp per segment (a run of <= kSegNodes nodes of one base cell) sums w_q r over
// its nodes; a node belongs to the cell holding it in its half-open box, clamped at the upper
// faces of the domain.  Lane sums, then a fixed shuffle tree.
__global__ void fine_restrict_cells_kernel(const float *r, int64_t r_ld, const int32_t *seg_ptr, const int32_t *cnode,
                                           const uint32_t *ccode, int nseg, int L, float *part, Cases cs) {
  pdl_begin();
  const int cc = case_of(cs, blockIdx.y);
  if (case_done(cs, cc)) return;
  r += cc * r_ld;
  part += (int64_t)cc * nseg * 24;
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= nseg) return;
  float acc[24];
#pragma unroll
  for (int q = 0; q < 24; ++q) acc[q] = 0.f;
  const int p1 = seg_ptr[warp + 1];
  for (int p = seg_ptr[warp] + lane; p < p1; p += 32) {
    const int n = cnode[p];
    const uint32_t cd = ccode[p];   // loaded beside n, not after it
    if (cd >> 31) continue;
    float w[8];
    trilinear8(cd, L, w);
    const float r0 = r[3 * (int64_t)n], r1 = r[3 * (int64_t)n + 1], r2 = r[3 * (int64_t)n + 2];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      acc[3 * q] = fmaf(w[q], r0, acc[3 * q]);
      acc[3 * q + 1] = fmaf(w[q], r1, acc[3 * q + 1]);
      acc[3 * q + 2] = fmaf(w[q], r2, acc[3 * q + 2]);
    }
  }
  // reduce-scatter over the warp: at each halving step a lane keeps the half of its sums that its
  // lane bit selects and adds its partner's copy of that half, so that lane l ends with the warp
  // total of sum l (16 + 8 + 4 + 2 + 1 shuffles instead of 24 x 5; sums 24..31 are zero)
  float v[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = q < 24 ? acc[q] : 0.f;
#pragma unroll
  for (int h = 16; h > 0; h >>= 1) {
    const bool upper = (lane & h) != 0;
#pragma unroll
    for (int q = 0; q < h; ++q) {
      const float keep = upper ? v[q + h] : v[q];
      const float send = upper ? v[q] : v[q + h];
      v[q] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  if (lane < 24) part[24 * (int64_t)warp + lane] = v[0];
}

// Stage 2: each level-0 DOF sums the partials of its <= 8 cells' segments (fixed order); with dinv
// also x = dinv b.
__global__ void __launch_bounds__(kT) fine_restrict_nodes_kernel(const float *part, int nseg, const int32_t *cseg,
                                                                 int X, int Y, int Z, unsigned faces, float *b,
                                                                 const float *dinv, float *x, Cases cs) {
  pdl_begin();
  const int cc = case_of(cs, blockIdx.y);
  if (case_done(cs, cc)) return;
  part += (int64_t)cc * nseg * 24;
  b += cc * lattice_len(X, Y, Z);
  if (x) x += cc * lattice_len(X, Y, Z);
  const int nodes = (X + 1) * (Y + 1) * (Z + 1);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nodes) return;
  const int J = t / 3, c = t % 3;
  const int i = J % (X + 1), j = (J / (X + 1)) % (Y + 1), k = J / ((X + 1) * (Y + 1));
  float s = 0.f;
  if (!lattice_fixed(i, j, k, X, Y, Z, faces)) {
    for (int cz = k - 1; cz <= k; ++cz) {
      if (cz < 0 || cz >= Z) continue;
      for (int cy = j - 1; cy <= j; ++cy) {
        if (cy < 0 || cy >= Y) continue;
        for (int cx = i - 1; cx <= i; ++cx) {
          if (cx < 0 || cx >= X) continue;
          const int q = (i - cx) + 2 * (j - cy) + 4 * (k - cz);
          const int cc = cx + X * (cy + Y * cz);
          for (int sg = cseg[cc]; sg < cseg[cc + 1]; ++sg) s += part[24 * (int64_t)sg + 3 * q + c];
        }
      }
    }
  }
  b[t] = s;
  if (x) x[t] = dinv[t] * s;
}

// (P0 v) at fine node n, component-wise into out[3].
__device__ __forceinline__ void prolong_at(const float *v, int cell, uint32_t cd, int L, int X, int Y, float out[3]) {
  float w[8];
  trilinear8(cd, L, w);
  const int cx = cell % X, cy = (cell / X) % Y, cz = cell / (X * Y);
  out[0] = out[1] = out[2] = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int J = (cx + (q & 1)) + (X + 1) * ((cy + ((q >> 1) & 1)) + (Y + 1) * (cz + (q >> 2)));
    out[0] = fmaf(w[q], v[3 * J], out[0]);
    out[1] = fmaf(w[q], v[3 * J + 1], out[1]);
    out[2] = fmaf(w[q], v[3 * J + 2], out[2]);
  }
}

// y = P0 v on the A-space (0 at constrained DOFs).
__global__ void fine_prolong_kernel(const float *v, const int32_t *ncell, const uint32_t *code, int64_t Nn, int L,
                                    int X, int Y, float *y) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < Nn; n += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t cd = code[n];
    float o[3] = {0.f, 0.f, 0.f};
    if (!(cd >> 31)) prolong_at(v, ncell[n], cd, L, X, Y, o);
    y[3 * n] = o[0]; y[3 * n + 1] = o[1]; y[3 * n + 2] = o[2];
  }
}

// b0 . x0 (per-CTA partials), then the last CTA finishes the preconditioned CG scalars:
//   mode 0 (iteration):  rz = rz_jacobi + b0.x0, beta = rz / rz_old
//   mode 1 (start):      rz = rz_jacobi + b0.x0
//   mode 2 (replacement): rz = rz_jacobi + b0.x0, beta = rz / prev, gamma = r.p / rz
// rz_jacobi = r^T D^-1 r is in scratch[0] (mode 0) or in rz (modes 1, 2); prev and r.p of a
// replacement are in scratch[2] and scratch[3].
__global__ void __launch_bounds__(kT) finish_kernel(const float *b0, const float *x0, int n, int mode,
                                                    SolveScalars *sc_all, int c0, double *partials_all,
                                                    int pstride, unsigned int *tickets) {
  pdl_begin();
  const int cc = c0 + blockIdx.y;
  SolveScalars *sc = sc_all + cc;
  if (sc->done) return;
  b0 += (int64_t)cc * n;
  x0 += (int64_t)cc * n;
  double *partials = partials_all + (int64_t)cc * pstride;
  unsigned int *ticket = tickets + cc;
  DotAcc<float> acc;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc.add_prod(b0[i], x0[i]);
  const double v = block_sum<kT>(acc.value());
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
  if (last_cta(ticket)) {
    const double bx = sum_partials<kT>(partials, gridDim.x);
    if (threadIdx.x == 0) {
      if (mode == 0) {
        const double rz = sc->scratch[0] + bx;
        sc->beta = rz / sc->rz;
        sc->rz_prev = sc->rz;
        sc->rz = rz;
      } else if (mode == 1) {
        sc->rz = sc->rz + bx;
      } else {
        const double rz = sc->rz + bx;
        sc->beta = rz / sc->scratch[2];
        sc->rp = sc->scratch[3] / rz;
        sc->rz = rz;
      }
      if (!isfinite(sc->rz) || !(sc->rz > 0.0) || !isfinite(sc->beta)) {
        sc->nonfinite = 1;
        sc->done = 1;
      }
    }
  }
}

// The search direction with the two-level preconditioner, z = D^-1 r + P0 x0:
//   mode 0: p = z + beta p;  mode 1: p = z;  mode 2: p = z + beta (p - gamma z).
__global__ void __launch_bounds__(kT) pupdate2_kernel(float *p, const float *r, int64_t ld, const float *dinv,
                                                      const float *x0, int64_t x0_ld, const int32_t *ncell,
                                                      const uint32_t *code, int64_t Nn, int L, int X, int Y, int mode,
                                                      const SolveScalars *sc_all, int c0) {
  pdl_begin();
  const int cc = c0 + blockIdx.y;
  const SolveScalars *sc = sc_all + cc;
  if (sc->done) return;
  p += cc * ld;
  r += cc * ld;
  x0 += cc * x0_ld;
  const float beta = (float)sc->beta, gamma = (float)sc->rp;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < Nn; n += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t cd = code[n];
    float pc[3] = {0.f, 0.f, 0.f};
    if (!(cd >> 31)) prolong_at(x0, ncell[n], cd, L, X, Y, pc);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t i = 3 * n + c;
      const float z = fmaf(dinv[i], r[i], pc[c]);
      if (mode == 0) p[i] = fmaf(beta, p[i], z);
      else if (mode == 1) p[i] = z;
      else p[i] = fmaf(beta, p[i] - gamma * z, z);
    }
  }
}

__global__ void first_sweep_kernel(const float *b, const float *dinv, float *x, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] = dinv[t] * b[t];
}

int grid_for(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t coarse_setup_launch(const DeviceMesh &m, CoarseHierarchy &h, const double *rho, cudaStream_t s) {
  const CoarseLevel &l0 = h.lev[0];
  const int nc0 = l0.X * l0.Y * l0.Z;
  moments0_kernel<<<grid_for(32 * (int64_t)nc0), kT, 0, s>>>(h.cell_elem, m.leaf, rho, nc0, l0.X, l0.Y, m.L, l0.H,
                                                             m.E0, m.Emin, m.penal, h.lev[0].mom);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int l = 1; l < h.nlev; ++l) {
    const CoarseLevel &c = h.lev[l];
    const CoarseLevel &f = h.lev[l - 1];
    moments_up_kernel<<<grid_for((int64_t)c.X * c.Y * c.Z), kT, 0, s>>>(f.mom, f.X, f.Y, f.Z, c.X, c.Y, c.Z, c.mom);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (int l = 0; l < h.nlev; ++l) {
    const CoarseLevel &c = h.lev[l];
    const int64_t n = (int64_t)c.X * c.Y * c.Z * kCellUpper;
    cellmat_kernel<<<grid_for(n), kT, 0, s>>>(c.mom, h.qent, h.qidx, h.qval, c.X * c.Y * c.Z, c.H, c.K,
                                              l == h.nlev - 1 ? h.Kc64 : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (l < h.nlev - 1) {
      l1diag_kernel<<<grid_for(c.nodes), kT, 0, s>>>(c.K, c.X, c.Y, c.Z, h.faces, c.dinv);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t coarse_restrict_launch(const DeviceMesh &m, const CoarseHierarchy &h, const float *r, int64_t r_ld,
                                   bool first_sweep, const SolveScalars *sc, int c0, int nv, cudaStream_t s) {
  const CoarseLevel &l0 = h.lev[0];
  const Cases cs{sc, c0};
  const dim3 g1(grid_for(32 * (int64_t)h.nseg), nv);
  { const cudaError_t pe_ = launch_pdl(fine_restrict_cells_kernel, dim3(g1), dim3(kT), 0, s, r, r_ld, h.seg_ptr, h.cnode, h.ccode, h.nseg, m.L, h.part, cs); if (pe_ != cudaSuccess) return pe_; }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool sweep = first_sweep && h.nlev > 1;
  const dim3 g2(grid_for(3 * (int64_t)l0.nodes), nv);
  { const cudaError_t pe_ = launch_pdl(fine_restrict_nodes_kernel, dim3(g2), dim3(kT), 0, s, h.part, h.nseg, h.cseg, l0.X, l0.Y, l0.Z, h.faces, l0.b,
                                               sweep ? l0.dinv : nullptr, sweep ? l0.x2 : nullptr, cs); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}

// V-cycle from level l with b_l given and (l not coarsest) the first sweep x = dinv_l b_l
// already in x2_l.  The remaining 2 nu - 1 sweeps alternate between x2 and x, so the result
// ends in x_l, where the next finer level's prolongation (or the fine level) reads it.
static cudaError_t vcycle_from(const CoarseHierarchy &h, int l, int nu, const Cases &cs, int nv, cudaStream_t s,
                               int *launches) {
  cudaError_t e;
  const CoarseLevel &c = h.lev[l];
  if (l == h.nlev - 1) {
    const int n = 3 * c.nodes;
    { const cudaError_t pe_ = launch_pdl(dense_solve_kernel, dim3(dim3((n + kDenseRows - 1) / kDenseRows, nv)), dim3(32 * kDenseRows), n * sizeof(float), s, 
        h.Ainv, c.b, c.x, n, cs); if (pe_ != cudaSuccess) return pe_; }
    *launches += 1;
    return cudaGetLastError();
  }
  const int n3 = 3 * c.nodes;
  const dim3 gl(grid_for(n3), nv), ga(grid_for(8 * (int64_t)n3), nv);
  float *cur = c.x2, *oth = c.x;
  for (int k = 1; k < nu; ++k) {           // remaining pre-smoothing sweeps
    { const cudaError_t pe_ = launch_pdl(level_apply_kernel, dim3(ga), dim3(kT), 0, s, c.K, cur, c.b, c.dinv, oth, c.X, c.Y, c.Z, h.faces, 1, cs); if (pe_ != cudaSuccess) return pe_; }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(cur, oth);
    *launches += 1;
  }
  { const cudaError_t pe_ = launch_pdl(level_apply_kernel, dim3(ga), dim3(kT), 0, s, c.K, cur, c.b, c.dinv, c.t, c.X, c.Y, c.Z, h.faces, 0, cs); if (pe_ != cudaSuccess) return pe_; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const CoarseLevel &n = h.lev[l + 1];
  const bool sweep = l + 1 < h.nlev - 1;
  const dim3 gn(grid_for(3 * (int64_t)n.nodes), nv);
  { const cudaError_t pe_ = launch_pdl(level_restrict_kernel, dim3(gn), dim3(kT), 0, s, c.t, c.X, c.Y, c.Z, n.X, n.Y, n.Z, h.faces, n.b, sweep ? n.dinv : nullptr,
                                          sweep ? n.x2 : nullptr, cs); if (pe_ != cudaSuccess) return pe_; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *launches += 2;
  if ((e = vcycle_from(h, l + 1, nu, cs, nv, s, launches)) != cudaSuccess) return e;
  { const cudaError_t pe_ = launch_pdl(level_prolong_kernel, dim3(gl), dim3(kT), 0, s, n.x, n.X, n.Y, n.Z, c.X, c.Y, c.Z, h.faces, cur, cs); if (pe_ != cudaSuccess) return pe_; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *launches += 1;
  for (int k = 0; k < nu; ++k) {
    { const cudaError_t pe_ = launch_pdl(level_apply_kernel, dim3(ga), dim3(kT), 0, s, c.K, cur, c.b, c.dinv, oth, c.X, c.Y, c.Z, h.faces, 1, cs); if (pe_ != cudaSuccess) return pe_; }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(cur, oth);
    *launches += 1;
  }
  return cur == c.x ? cudaSuccess : cudaErrorInvalidValue;   // 2 nu - 1 sweeps: always x
}

cudaError_t coarse_vcycle_launch(const CoarseHierarchy &h, int nu, const SolveScalars *sc, int c0, int nv,
                                 cudaStream_t s, int *launches) {
  return vcycle_from(h, 0, nu, Cases{sc, c0}, nv, s, launches);
}

cudaError_t coarse_finish_launch(const CoarseHierarchy &h, int mode, SolveScalars *sc, int c0, int nv,
                                 double *partials, int pstride, unsigned int *tickets, cudaStream_t s) {
  const int n = 3 * h.lev[0].nodes;
  int g = grid_for(n);
  if (g > 4 * device_sms()) g = 4 * device_sms();   // one grid for every caller: the same reduction order
  if (g > pstride) return cudaErrorInvalidValue;
  { const cudaError_t pe_ = launch_pdl(finish_kernel, dim3(dim3(g, nv)), dim3(kT), 0, s, h.lev[0].b, h.lev[0].x, n, mode, sc, c0, partials, pstride, tickets); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}

cudaError_t coarse_pupdate_launch(const DeviceMesh &m, const CoarseHierarchy &h, float *p, const float *r,
                                  int64_t ld, const float *dinv, int mode, const SolveScalars *sc, int c0, int nv,
                                  cudaStream_t s) {
  int g = grid_for(m.Nn);
  if (g > 8 * device_sms()) g = 8 * device_sms();
  { const cudaError_t pe_ = launch_pdl(pupdate2_kernel, dim3(dim3(g, nv)), dim3(kT), 0, s, p, r, ld, dinv, h.lev[0].x, 3 * (int64_t)h.lev[0].nodes, h.ncell, h.code,
                                             m.Nn, m.L, h.lev[0].X, h.lev[0].Y, mode, sc, c0); if (pe_ != cudaSuccess) return pe_; }
  return cudaGetLastError();
}

cudaError_t coarse_prolong_launch(const DeviceMesh &m, const CoarseHierarchy &h, const float *v, float *y,
                                  cudaStream_t s) {
  int g = grid_for(m.Nn);
  if (g > 8 * device_sms()) g = 8 * device_sms();
  fine_prolong_kernel<<<g, kT, 0, s>>>(v, h.ncell, h.code, m.Nn, m.L, h.lev[0].X, h.lev[0].Y, y);
  return cudaGetLastError();
}

// x2_0 = dinv_0 b_0: the first sweep of a cycle whose level-0 right-hand side was set directly.
cudaError_t coarse_first_sweep_launch(const CoarseHierarchy &h, cudaStream_t s) {
  if (h.nlev < 2) return cudaSuccess;
  const CoarseLevel &c = h.lev[0];
  first_sweep_kernel<<<grid_for(3 * (int64_t)c.nodes), kT, 0, s>>>(c.b, c.dinv, c.x2, 3 * c.nodes);
  return cudaGetLastError();
}

cudaError_t coarse_level_apply_launch(const CoarseHierarchy &h, int l, const float *x, float *y, cudaStream_t s) {
  const CoarseLevel &c = h.lev[l];
  level_apply_kernel<<<grid_for(24 * (int64_t)c.nodes), kT, 0, s>>>(c.K, x, nullptr, c.dinv, y, c.X, c.Y, c.Z, h.faces,
                                                                    2, Cases{nullptr, 0});
  return cudaGetLastError();
}

}  // namespace amr
