// Host tables of the two-level preconditioner (kernels_coarse.cu): the level shapes, which
// leaves and mesh nodes belong to which base cell, the moment matrices Q_abc of the cell basis
// and the dense inverse of the coarsest level.  Integer work and small dense algebra only.
#include <algorithm>
#include <cmath>
#include <exception>
#include <thread>
#include <string>
#include <vector>

#include "tm_internal.h"

namespace amr {

// f(t, lo, hi) over nt contiguous chunks of [0, n) on host threads (host_thread_limit(), one per
// 64k items, and so that the threads' per_thread_ints int32 each stay within 256 MB).  A chunk
// whose thread cannot be started runs on the calling thread; an exception is rethrown after the
// join.
static int parallel_chunks_threads(int64_t n, int64_t per_thread_ints = 0) {
  int64_t nt = std::min<int64_t>(host_thread_limit(), n / 65536 + 1);
  if (per_thread_ints > 0) nt = std::min<int64_t>(nt, std::max<int64_t>(1, ((int64_t)1 << 26) / per_thread_ints));
  return (int)std::max<int64_t>(1, nt);
}

template <typename F>
static void parallel_chunks(int64_t n, F f, int nt = 0) {
  if (nt <= 0) nt = parallel_chunks_threads(n);
  std::vector<std::exception_ptr> ex(nt);
  auto run = [&](int t) {
    try {
      f(t, n * t / nt, n * (t + 1) / nt);
    } catch (...) {
      ex[t] = std::current_exception();
    }
  };
  std::vector<std::thread> pool;
  std::vector<int> here;
  pool.reserve(nt);
  here.reserve(nt);
  for (int t = 1; t < nt; ++t) {
    try {
      pool.emplace_back(run, t);
    } catch (...) {
      here.push_back(t);
    }
  }
  run(0);
  for (int t : here) run(t);
  for (auto &th : pool) th.join();
  for (const std::exception_ptr &e : ex)
    if (e) std::rethrow_exception(e);
}

// Level 0 is the base grid; level l+1 has ceil(n / 2) cells per axis for the n of level l (a
// coarse cell may overhang the box: the coarse functions restricted to the box stay nested),
// added while level l has more than 64 cells.  An axis whose upper face is clamped is halved
// only while its count is even (the clamped face stays a lattice plane).
std::string coarse_shapes(const HostMesh &m, std::vector<int> &shapes) {
  shapes.clear();
  if (m.L > 9) return "node positions in a base cell need max_level <= 9";
  int d[3] = {m.nx, m.ny, m.nz};
  shapes.insert(shapes.end(), {d[0], d[1], d[2]});
  while ((int64_t)d[0] * d[1] * d[2] > 64 && (int)shapes.size() / 3 < kMaxCoarseLevels) {
    bool stop = false;
    for (int a = 0; a < 3; ++a)
      if ((d[a] % 2) && ((m.dirichlet_faces >> (2 * a + 1)) & 1u)) stop = true;
    if (stop) break;
    for (int a = 0; a < 3; ++a) d[a] = (d[a] + 1) / 2;
    shapes.insert(shapes.end(), {d[0], d[1], d[2]});
  }
  int X, Y, Z;
  const int n = (int)shapes.size() / 3;
  X = shapes[3 * (n - 1)]; Y = shapes[3 * (n - 1) + 1]; Z = shapes[3 * (n - 1) + 2];
  const int64_t dofs = 3 * (int64_t)(X + 1) * (Y + 1) * (Z + 1);
  if (dofs > kMaxCoarsestDofs)
    return "the base grid " + std::to_string(m.nx) + "x" + std::to_string(m.ny) + "x" + std::to_string(m.nz) +
           " halves only down to " + std::to_string(X) + "x" + std::to_string(Y) + "x" + std::to_string(Z) +
           " cells (" + std::to_string(dofs) + " coarsest unknowns, at most " + std::to_string(kMaxCoarsestDofs) +
           " are solved directly)";
  return "";
}

// cell_elem: per base cell (x fastest) the canonical range of its leaves (contiguous in Morton
// order).  cptr/cnode: per base cell the mesh nodes it owns, i.e. those in its half-open box,
// the box closed at the upper faces of the domain.  ncell/code: per node its owning cell and its
// position there (finest units, 10 bits per axis) with bit 31 set for hanging or clamped nodes.
void coarse_tables(const HostMesh &m, std::vector<int32_t> &cell_elem, std::vector<int32_t> &cptr,
                   std::vector<int32_t> &cnode, std::vector<int32_t> &ncell, std::vector<uint32_t> &code) {
  const int X = m.nx, Y = m.ny, Z = m.nz, S = 1 << m.L;
  const int64_t ncells = (int64_t)X * Y * Z;
  // a base cell's leaves are one run of the Morton order: each run's ends are found where the
  // neighbouring leaf lies in another cell, independently per leaf
  auto cell_of = [&](int64_t e) {
    const int32_t *l = &m.leaf[4 * e];
    return (l[0] / S) + X * ((l[1] / S) + (int64_t)Y * (l[2] / S));
  };
  cell_elem.assign(2 * ncells, 0);
  parallel_chunks(m.Ne, [&](int, int64_t lo, int64_t hi) {
    for (int64_t e = lo; e < hi; ++e) {
      const int64_t c = cell_of(e);
      if (e == 0 || cell_of(e - 1) != c) cell_elem[2 * c] = (int32_t)e;
      if (e + 1 == m.Ne || cell_of(e + 1) != c) cell_elem[2 * c + 1] = (int32_t)(e + 1);
    }
  });
  // nodes by owning cell, ascending within a cell: per chunk of nodes its cell counts, then each
  // chunk fills its nodes after the earlier chunks' nodes of the same cell
  ncell.assign(m.Nn, 0);
  code.assign(m.Nn, 0);
  const int nt = parallel_chunks_threads(m.Nn, ncells);
  std::vector<int32_t> cnt((size_t)nt * ncells, 0);
  parallel_chunks(m.Nn, [&](int t, int64_t lo, int64_t hi) {
    int32_t *ct = &cnt[(size_t)t * ncells];
    for (int64_t n = lo; n < hi; ++n) {
      const int32_t *p = &m.node_xyz[3 * n];
      const int cx = std::min(p[0] / S, X - 1), cy = std::min(p[1] / S, Y - 1), cz = std::min(p[2] / S, Z - 1);
      const int64_t c = cx + X * (cy + (int64_t)Y * cz);
      ncell[n] = (int32_t)c;
      uint32_t cd = (uint32_t)(p[0] - cx * S) | ((uint32_t)(p[1] - cy * S) << 10) | ((uint32_t)(p[2] - cz * S) << 20);
      if (m.nflag[n]) cd |= 0x80000000u;
      code[n] = cd;
      ct[c]++;
    }
  }, nt);
  cptr.assign(ncells + 1, 0);
  for (int64_t c = 0; c < ncells; ++c) {
    int32_t run = cptr[c];
    for (int t = 0; t < nt; ++t) {
      const int32_t v = cnt[(size_t)t * ncells + c];
      cnt[(size_t)t * ncells + c] = run;
      run += v;
    }
    cptr[c + 1] = run;
  }
  cnode.assign(m.Nn, 0);
  parallel_chunks(m.Nn, [&](int t, int64_t lo, int64_t hi) {
    int32_t *fill = &cnt[(size_t)t * ncells];
    for (int64_t n = lo; n < hi; ++n) cnode[fill[ncell[n]]++] = (int32_t)n;
  }, nt);
}

// Segments of the restriction: each cell's node run cut into pieces of at most kSegNodes, so
// that one warp per segment has balanced work (cells hold 8 to (2^L + 1)^3 nodes).
void coarse_segments(const std::vector<int32_t> &cptr, std::vector<int32_t> &seg_ptr, std::vector<int32_t> &seg_cell,
                     std::vector<int32_t> &cseg) {
  const int64_t ncells = (int64_t)cptr.size() - 1;
  seg_ptr.clear();
  seg_cell.clear();
  cseg.assign(ncells + 1, 0);
  for (int64_t c = 0; c < ncells; ++c) {
    cseg[c] = (int32_t)seg_cell.size();
    for (int32_t p = cptr[c]; p < cptr[c + 1]; p += kSegNodes) {
      seg_ptr.push_back(p);
      seg_cell.push_back((int32_t)c);
    }
  }
  cseg[ncells] = (int32_t)seg_cell.size();
  seg_ptr.push_back(cptr[ncells]);
}

// Q_abc (27 x 576, entry (3 I + c) * 24 + 3 J + c'): the coefficient of s_x^a s_y^b s_z^c in the
// D-weighted product of the centred-coordinate gradients of the cell basis functions I and J,
//   sum over alpha, beta of M[c][c'][alpha][beta] d_alpha phi_I d_beta phi_J,
// with phi_I(s) = prod_a (1 + sigma_a s_a) / 2 and M the contraction of the isotropic D (E = 1)
// with the strain-displacement pattern (Voigt order xx, yy, zz, xy, yz, zx).
void coarse_moment_matrices(double nu, std::vector<double> &Q) {
  const double lam = nu / ((1 + nu) * (1 - 2 * nu)), mu = 1.0 / (2 * (1 + nu));
  double D[6][6] = {};
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) D[p][q] = lam;
  for (int p = 0; p < 3; ++p) D[p][p] = lam + 2 * mu;
  for (int p = 3; p < 6; ++p) D[p][p] = mu;
  // G[p][c][alpha]: strain p = sum over (c, alpha) of G * d_alpha u_c
  double G[6][3][3] = {};
  G[0][0][0] = 1; G[1][1][1] = 1; G[2][2][2] = 1;
  G[3][0][1] = 1; G[3][1][0] = 1;
  G[4][1][2] = 1; G[4][2][1] = 1;
  G[5][0][2] = 1; G[5][2][0] = 1;
  double M[3][3][3][3] = {};
  for (int c = 0; c < 3; ++c)
    for (int c2 = 0; c2 < 3; ++c2)
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) {
          double s = 0;
          for (int p = 0; p < 6; ++p)
            for (int q = 0; q < 6; ++q) s += G[p][c][al] * D[p][q] * G[q][c2][be];
          M[c][c2][al][be] = s;
        }
  // 1D factor of d_alpha phi_I along axis a as a polynomial (c0, c1) in s
  auto factor = [](int I, int a, int alpha, double out[2]) {
    const double sg = ((I >> a) & 1) ? 1.0 : -1.0;
    if (a == alpha) { out[0] = sg / 2; out[1] = 0; }
    else { out[0] = 0.5; out[1] = sg / 2; }
  };
  Q.assign(27 * 576, 0.0);
  for (int I = 0; I < 8; ++I)
    for (int J = 0; J < 8; ++J)
      for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) {
          double P[3][3];   // per axis, coefficients of s^0, s^1, s^2 of the product
          for (int a = 0; a < 3; ++a) {
            double f[2], g[2];
            factor(I, a, al, f);
            factor(J, a, be, g);
            P[a][0] = f[0] * g[0];
            P[a][1] = f[0] * g[1] + f[1] * g[0];
            P[a][2] = f[1] * g[1];
          }
          for (int c = 0; c < 3; ++c)
            for (int c2 = 0; c2 < 3; ++c2) {
              const double w = M[c][c2][al][be];
              if (w == 0) continue;
              const int ent = (3 * I + c) * 24 + 3 * J + c2;
              for (int z = 0; z < 3; ++z)
                for (int y = 0; y < 3; ++y)
                  for (int x = 0; x < 3; ++x) Q[(x + 3 * y + 9 * z) * 576 + ent] += w * P[0][x] * P[1][y] * P[2][z];
            }
        }
}

// Dense inverse of the coarsest level's matrix (assembled from its FP64 cell matrices over the
// free DOFs) by Cholesky factorisation; returned over all 3 (X+1)(Y+1)(Z+1) DOFs, with zero rows
// and columns at clamped nodes.
// a . b over n entries with four interleaved partial sums (a fixed order the compiler can vectorize)
static double dot4(const double *a, const double *b, int n) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int k = 0;
  for (; k + 4 <= n; k += 4) {
    s0 += a[k] * b[k];
    s1 += a[k + 1] * b[k + 1];
    s2 += a[k + 2] * b[k + 2];
    s3 += a[k + 3] * b[k + 3];
  }
  for (; k < n; ++k) s0 += a[k] * b[k];
  return (s0 + s1) + (s2 + s3);
}

// f(i) for i in [0, n) on up to 8 host threads, rows dealt out round robin (row costs fall with i).
// A stripe whose thread cannot be started runs on the calling thread; an exception is caught on
// its thread and rethrown here once every thread has joined.
template <typename F>
static void parallel_rows(int n, F f) {
  const int nt = std::max(1, std::min({8, host_thread_limit(), n / 32}));
  std::vector<std::exception_ptr> ex(nt);
  auto stripe = [&](int t) {
    try {
      for (int i = t; i < n; i += nt) f(i);
    } catch (...) {
      ex[t] = std::current_exception();
    }
  };
  std::vector<std::thread> pool;
  std::vector<int> here;
  pool.reserve(nt);
  here.reserve(nt);
  for (int t = 1; t < nt; ++t) {
    try {
      pool.emplace_back(stripe, t);
    } catch (...) {
      here.push_back(t);
    }
  }
  stripe(0);
  for (int t : here) stripe(t);
  for (auto &th : pool) th.join();
  for (const std::exception_ptr &e : ex)
    if (e) std::rethrow_exception(e);
}

std::string coarse_dense_inverse(const std::vector<double> &Kc, int X, int Y, int Z, unsigned faces,
                                 std::vector<float> &Ainv) {
  const int nodes = (X + 1) * (Y + 1) * (Z + 1), n = 3 * nodes;
  auto fixed = [&](int i, int j, int k) {
    return ((faces & 1u) && i == 0) || ((faces & 2u) && i == X) || ((faces & 4u) && j == 0) ||
           ((faces & 8u) && j == Y) || ((faces & 16u) && k == 0) || ((faces & 32u) && k == Z);
  };
  std::vector<int> fmap(n, -1);
  int nf = 0;
  for (int I = 0; I < nodes; ++I) {
    const int i = I % (X + 1), j = (I / (X + 1)) % (Y + 1), k = I / ((X + 1) * (Y + 1));
    if (!fixed(i, j, k))
      for (int c = 0; c < 3; ++c) fmap[3 * I + c] = nf++;
  }
  std::vector<double> A((size_t)nf * nf, 0.0);
  for (int cz = 0; cz < Z; ++cz)
    for (int cy = 0; cy < Y; ++cy)
      for (int cx = 0; cx < X; ++cx) {
        const double *K = &Kc[576 * (size_t)(cx + X * (cy + Y * cz))];
        int dof[24];
        for (int q = 0; q < 8; ++q) {
          const int I = (cx + (q & 1)) + (X + 1) * ((cy + ((q >> 1) & 1)) + (Y + 1) * (cz + (q >> 2)));
          for (int c = 0; c < 3; ++c) dof[3 * q + c] = fmap[3 * I + c];
        }
        for (int r = 0; r < 24; ++r)
          if (dof[r] >= 0)
            for (int s = 0; s < 24; ++s)
              if (dof[s] >= 0) A[(size_t)dof[r] * nf + dof[s]] += K[r * 24 + s];
      }
  // Cholesky A = L L^T (lower triangle in place), rows of L contiguous
  for (int j = 0; j < nf; ++j) {
    const double *lj = &A[(size_t)j * nf];
    const double d = A[(size_t)j * nf + j] - dot4(lj, lj, j);
    if (!(d > 0)) return "the coarsest level's matrix is not positive definite";
    const double ljj = std::sqrt(d);
    A[(size_t)j * nf + j] = ljj;
    for (int i = j + 1; i < nf; ++i) {
      const double *li = &A[(size_t)i * nf];
      A[(size_t)i * nf + j] = (A[(size_t)i * nf + j] - dot4(li, lj, j)) / ljj;
    }
  }
  // Yt = (L^-1)^T, one column of L^-1 per row of Yt: forward substitution with e_c, entries
  // below c only; then A^-1 = Yt Yt^T restricted to the lower triangle and mirrored.  The columns
  // and the rows of the product are independent: they are spread over host threads, each entry
  // computed by one thread in a fixed order (the result does not depend on the thread count).
  std::vector<double> Yt((size_t)nf * nf, 0.0), inv((size_t)nf * nf, 0.0);
  parallel_rows(nf, [&](int c) {
    double *y = &Yt[(size_t)c * nf];
    y[c] = 1.0 / A[(size_t)c * nf + c];
    for (int i = c + 1; i < nf; ++i) {
      const double *li = &A[(size_t)i * nf];
      y[i] = -dot4(li + c, y + c, i - c) / li[i];
    }
  });
  parallel_rows(nf, [&](int r) {
    const double *yr = &Yt[(size_t)r * nf];
    for (int c = 0; c <= r; ++c) inv[(size_t)r * nf + c] = dot4(yr + r, &Yt[(size_t)c * nf] + r, nf - r);
  });
  for (int r = 0; r < nf; ++r)
    for (int c = r + 1; c < nf; ++c) inv[(size_t)r * nf + c] = inv[(size_t)c * nf + r];
  Ainv.assign((size_t)n * n, 0.f);
  for (int r = 0; r < n; ++r)
    if (fmap[r] >= 0)
      for (int s = 0; s < n; ++s)
        if (fmap[s] >= 0) Ainv[(size_t)r * n + s] = (float)(0.5 * (inv[(size_t)fmap[r] * nf + fmap[s]] +
                                                                    inv[(size_t)fmap[s] * nf + fmap[r]]));
  return "";
}

}  // namespace amr
