// Host construction of the mesh tables of paper Sec. 6 (hanging-node
// interpolation, Eq. 6) for a 2:1-balanced octree leaf set, plus the block,
// colour and diagonal tables the device kernels use.  Integer work only
// (except the reference element matrix and the diagonal coefficient table).
//
// Algorithm (independent of any other implementation in this repository):
//  1. leaves sorted by Morton key with an LSD radix sort; aligned octants occupy
//     contiguous Morton intervals, so disjointness is "each interval ends before
//     the next begins" and coverage is "the lengths add up to the box";
//  2. nodes = radix-sorted unique corner keys;
//  3. balance = for every node, the leaves owning the <= 8 finest cells around it
//     differ by at most one level (dense finest-grid owner map);
//  4. on a balanced mesh a node hangs exactly when it is the midpoint of a leaf
//     edge (masters: the edge ends, weight 1/2) or the centre of a leaf face
//     (masters: the face corners, weight 1/4); each leaf probes its 12 edge
//     midpoints and 6 face centres against the node set.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <unordered_map>
#include <memory>
#include <numeric>
#include <thread>

#include "tm_internal.h"

namespace amr {

static inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// the inverse of spread3: bits 0, 3, 6, ... of x packed together
static inline uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x | (x >> 4)) & 0x100f00f00f00f00full;
  x = (x | (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x | (x >> 16)) & 0x1f00000000ffffull;
  x = (x | (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

// LSD radix sort of keys, returning the permutation (stable).
static_assert(kBlockElems * kSlotRow < kQuarterBit, "inverse-list slot offsets must stay below the fold bits");

// The tables keep node ids and their list, slot and record offsets in 32-bit integers; a mesh
// whose tables would need more is rejected.
constexpr int64_t kMaxOffset = ((int64_t)1 << 31) - 1;
constexpr const char *kTooLarge = "mesh too large: a table offset would exceed 2^31 - 1";

// Host threads for the table builds: host_thread_limit(), at most one per 64k items.  The tables
// do not depend on the number.
static int host_threads(size_t n) {
  return (int)std::max<size_t>(1, std::min<size_t>((size_t)host_thread_limit(), n / 65536 + 1));
}

// A chunk whose thread cannot be started runs on the calling thread (the chunks share nothing but
// their index t, so where they run does not change the result), and an exception a chunk throws
// is caught on its thread and rethrown here once every thread has joined.
template <typename F>
static void chunked(int nt, size_t n, F f) {
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

// Each pass: per-chunk digit counts, then every chunk scatters its items in order to the positions
// the counts of the lower digits and of the earlier chunks leave free -- the sequential stable
// order, whatever the number of threads.
static std::vector<int64_t> radix_order(const std::vector<uint64_t> &key, std::vector<uint64_t> *sorted = nullptr) {
  const size_t n = key.size();
  uint64_t mx = 0;
  for (uint64_t k : key) mx |= k;
  int bits = 0;
  while (bits < 64 && (mx >> bits)) ++bits;
  // keys travel with their indices, so every pass streams both arrays in order
  std::vector<uint32_t> idx(n), tmp(n);
  std::vector<uint64_t> k(key), ktmp(n);
  std::iota(idx.begin(), idx.end(), 0u);
  const int R = 11, B = 1 << R;
  const int nt = host_threads(n);
  std::vector<size_t> cnt((size_t)nt * B);
  for (int sh = 0; sh < bits; sh += R) {
    chunked(nt, n, [&](int t, size_t lo, size_t hi) {
      size_t *c = &cnt[(size_t)t * B];
      std::fill(c, c + B, 0);
      for (size_t i = lo; i < hi; ++i) c[(k[i] >> sh) & (B - 1)]++;
    });
    size_t run = 0;   // digit-major, chunk-minor exclusive prefix
    for (int d = 0; d < B; ++d)
      for (int t = 0; t < nt; ++t) {
        const size_t v = cnt[(size_t)t * B + d];
        cnt[(size_t)t * B + d] = run;
        run += v;
      }
    chunked(nt, n, [&](int t, size_t lo, size_t hi) {
      size_t *c = &cnt[(size_t)t * B];
      for (size_t i = lo; i < hi; ++i) {
        const size_t d = c[(k[i] >> sh) & (B - 1)]++;
        tmp[d] = idx[i];
        ktmp[d] = k[i];
      }
    });
    idx.swap(tmp);
    k.swap(ktmp);
  }
  if (sorted) sorted->swap(k);
  return std::vector<int64_t>(idx.begin(), idx.end());
}

void reference_stiffness(double nu, double *K0) {
  // K0 = sum over 2x2x2 Gauss points of B^T D B / 8 on the unit cube, E = 1.
  const double lam = nu / ((1 + nu) * (1 - 2 * nu)), mu = 0.5 / (1 + nu);
  double D[6][6] = {};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) D[a][b] = lam + (a == b ? 2 * mu : 0);
  D[3][3] = D[4][4] = D[5][5] = mu;
  const double g = 1.0 / std::sqrt(3.0);
  const double pts[2] = {0.5 * (1 - g), 0.5 * (1 + g)};
  std::fill(K0, K0 + 576, 0.0);
  for (int qa = 0; qa < 2; ++qa)
    for (int qb = 0; qb < 2; ++qb)
      for (int qc = 0; qc < 2; ++qc) {
        const double xi[3] = {pts[qa], pts[qb], pts[qc]};
        double B[6][24] = {};
        for (int k = 0; k < 8; ++k) {
          const int i = k & 1, j = (k >> 1) & 1, m = (k >> 2) & 1;
          const double f0 = i ? xi[0] : 1 - xi[0], f1 = j ? xi[1] : 1 - xi[1], f2 = m ? xi[2] : 1 - xi[2];
          const double d0 = i ? 1 : -1, d1 = j ? 1 : -1, d2 = m ? 1 : -1;
          const double gx = d0 * f1 * f2, gy = f0 * d1 * f2, gz = f0 * f1 * d2;
          B[0][3 * k] = gx;
          B[1][3 * k + 1] = gy;
          B[2][3 * k + 2] = gz;
          B[3][3 * k] = gy;
          B[3][3 * k + 1] = gx;
          B[4][3 * k + 1] = gz;
          B[4][3 * k + 2] = gy;
          B[5][3 * k] = gz;
          B[5][3 * k + 2] = gx;
        }
        double DB[6][24];
        for (int a = 0; a < 6; ++a)
          for (int c = 0; c < 24; ++c) {
            double s = 0;
            for (int b = 0; b < 6; ++b) s += D[a][b] * B[b][c];
            DB[a][c] = s;
          }
        for (int r = 0; r < 24; ++r)
          for (int c = 0; c < 24; ++c) {
            double s = 0;
            for (int a = 0; a < 6; ++a) s += B[a][r] * DB[a][c];
            K0[r * 24 + c] += 0.125 * s;
          }
      }
}

static inline int64_t find_key(const std::vector<uint64_t> &keys, uint64_t k) {
  auto it = std::lower_bound(keys.begin(), keys.end(), k);
  if (it == keys.end() || *it != k) return -1;
  return it - keys.begin();
}

std::string build_host_mesh(const tm_mesh_desc &d, HostMesh &m) {
  m = HostMesh();
  if (d.nx < 1 || d.ny < 1 || d.nz < 1) return "base grid must be at least 1x1x1";
  if (d.max_level < 0 || d.max_level > 12) return "max_level must be in [0, 12]";
  if (!(d.h0 > 0)) return "h0 must be positive";
  if (d.n_leaves < 1 || !d.leaves) return "no leaves";
  if (d.n_leaves >= (int64_t)1 << 29) return "more than 2^29 - 1 leaves";   // 8 corners each, 32-bit sort indices
  if (!(d.nu > -1.0 && d.nu < 0.5)) return "Poisson ratio must be in (-1, 0.5)";
  if (!(d.E0 > d.Emin && d.Emin >= 0)) return "need E0 > Emin >= 0";
  if (!(d.penal >= 1)) return "penalty must be >= 1";
  const int L = d.max_level;
  const int64_t fx = (int64_t)d.nx << L, fy = (int64_t)d.ny << L, fz = (int64_t)d.nz << L;
  if (fx >= (1 << 20) || fy >= (1 << 20) || fz >= (1 << 20)) return "finest grid too large";
  if (fx * fy * fz > (int64_t)1 << 31) return "finest grid has more than 2^31 cells";
  m.nx = d.nx; m.ny = d.ny; m.nz = d.nz; m.L = L; m.h0 = d.h0;
  m.dirichlet_faces = d.dirichlet_faces;
  m.E0 = d.E0; m.Emin = d.Emin; m.nu = d.nu; m.penal = d.penal;
  const int64_t Ne = d.n_leaves;
  m.Ne = Ne;

  // ---- 1. validate, sort, disjoint + cover (on host threads: the first failing leaf of the first
  // failing chunk is the first failing leaf in order)
  std::vector<uint64_t> key(Ne);
  {
    const int nt = host_threads(Ne);
    std::vector<const char *> err(nt, nullptr);
    chunked(nt, (size_t)Ne, [&](int t, size_t lo, size_t hi) {
      for (size_t e = lo; e < hi; ++e) {
        const int32_t *l = d.leaves + 4 * e;
        if (l[3] < 0 || l[3] > L) { err[t] = "leaf level out of range"; return; }
        const int64_t s = (int64_t)1 << (L - l[3]);
        for (int a = 0; a < 3; ++a) {
          const int64_t ext = a == 0 ? fx : (a == 1 ? fy : fz);
          if (l[a] < 0 || l[a] + s > ext) { err[t] = "leaf outside the domain"; return; }
          if (l[a] % s) { err[t] = "leaf anchor not aligned to its size"; return; }
        }
        key[e] = morton3(l[0], l[1], l[2]);
      }
    });
    for (const char *e : err)
      if (e) return e;
  }
  m.perm = radix_order(key);
  m.leaf.resize(4 * Ne);
  {
    // sorted leaves that each end at or before the next one's key neither overlap nor, when their
    // volumes add up to the domain's, leave a gap
    const int nt = host_threads(Ne);
    std::vector<int64_t> covered(nt, 0);
    std::vector<uint8_t> overlap(nt, 0);
    chunked(nt, (size_t)Ne, [&](int t, size_t lo, size_t hi) {
      for (size_t i = lo; i < hi; ++i) {
        const int32_t *l = d.leaves + 4 * m.perm[i];
        std::memcpy(&m.leaf[4 * i], l, 16);
        const int64_t s = (int64_t)1 << (L - l[3]);
        covered[t] += s * s * s;
        if ((int64_t)i + 1 < Ne && key[m.perm[i]] + (uint64_t)(s * s * s) > key[m.perm[i + 1]]) overlap[t] = 1;
      }
    });
    int64_t total = 0;
    for (int t = 0; t < nt; ++t) {
      if (overlap[t]) return "leaves overlap";
      total += covered[t];
    }
    if (total != fx * fy * fz) return "leaves do not cover the domain";
  }

  // ---- 2. nodes: the distinct corner keys in Morton order; conn and coordinates from them
  auto corner_key = [&](size_t e, int k) {
    const int32_t *l = &m.leaf[4 * e];
    const int32_t s = 1 << (L - l[3]);
    return morton3(l[0] + s * (k & 1), l[1] + s * ((k >> 1) & 1), l[2] + s * ((k >> 2) & 1));
  };
  // the key grows with each coordinate, so the domain's far corner (always a node) has the
  // largest key
  const uint64_t nword = morton3((uint32_t)fx, (uint32_t)fy, (uint32_t)fz) / 64 + 1;
  // a bitmap of the Morton key space (when it is small enough): a node's id is the number of
  // distinct corner keys below its own, the same numbering as sorting and deduplicating the keys
  std::vector<uint64_t> bm;
  std::vector<int64_t> below;   // set bits in the words before w
  if (nword <= std::max<uint64_t>(1u << 16, (uint64_t)(8 * Ne))) {
    bm.assign(nword, 0);
    chunked(host_threads(8 * Ne), (size_t)Ne, [&](int, size_t lo, size_t hi) {
      for (size_t e = lo; e < hi; ++e)
        for (int k = 0; k < 8; ++k) {
          const uint64_t ck = corner_key(e, k);
          uint64_t *w = &bm[ck >> 6];
          const uint64_t b = 1ull << (ck & 63);
          if (!(__atomic_load_n(w, __ATOMIC_RELAXED) & b)) __atomic_fetch_or(w, b, __ATOMIC_RELAXED);
        }
    });
    below.resize(nword);
    const int nt = host_threads(nword * 8);
    std::vector<int64_t> part(nt + 1, 0);
    chunked(nt, nword, [&](int t, size_t lo, size_t hi) {
      int64_t c = 0;
      for (size_t w = lo; w < hi; ++w) c += __builtin_popcountll(bm[w]);
      part[t + 1] = c;
    });
    for (int t = 0; t < nt; ++t) part[t + 1] += part[t];
    m.Nn = part[nt];
    m.node_key.resize(m.Nn);
    chunked(nt, nword, [&](int t, size_t lo, size_t hi) {
      int64_t c = part[t];
      for (size_t w = lo; w < hi; ++w) {
        below[w] = c;
        for (uint64_t v = bm[w]; v; v &= v - 1) m.node_key[c++] = 64 * (uint64_t)w + __builtin_ctzll(v);
      }
    });
    m.conn.resize(8 * Ne);
    chunked(host_threads(8 * Ne), (size_t)Ne, [&](int, size_t lo, size_t hi) {
      for (size_t e = lo; e < hi; ++e)
        for (int k = 0; k < 8; ++k) {
          const uint64_t ck = corner_key(e, k);
          const uint64_t w = ck >> 6, low = (1ull << (ck & 63)) - 1;
          m.conn[8 * e + k] = (int32_t)(below[w] + __builtin_popcountll(bm[w] & low));
        }
    });
  } else {
    std::vector<uint64_t> ckey(8 * Ne);
    chunked(host_threads(Ne), (size_t)Ne, [&](int, size_t lo, size_t hi) {
      for (size_t e = lo; e < hi; ++e)
        for (int k = 0; k < 8; ++k) ckey[8 * e + k] = corner_key(e, k);
    });
    std::vector<uint64_t> sk;
    const std::vector<int64_t> ord = radix_order(ckey, &sk);
    std::vector<int32_t> nid(8 * Ne);
    int64_t nn = -1;
    uint64_t prev = ~0ull;
    for (int64_t i = 0; i < 8 * Ne; ++i) {
      if (sk[i] != prev) {
        ++nn;
        m.node_key.push_back(sk[i]);
        prev = sk[i];
      }
      nid[i] = (int32_t)nn;
    }
    m.Nn = nn + 1;
    m.conn.resize(8 * Ne);
    chunked(host_threads(8 * Ne), (size_t)(8 * Ne), [&](int, size_t lo, size_t hi) {
      for (size_t i = lo; i < hi; ++i) m.conn[ord[i]] = nid[i];
    });
  }
  if (3 * m.Nn > kMaxOffset) return kTooLarge;   // 3 DOFs per node
  const int64_t Nn = m.Nn;
  m.node_xyz.resize(3 * Nn);
  chunked(host_threads(Nn), (size_t)Nn, [&](int, size_t lo, size_t hi) {
    for (size_t n = lo; n < hi; ++n) {
      const uint64_t k = m.node_key[n];
      m.node_xyz[3 * n] = (int32_t)compact3(k);
      m.node_xyz[3 * n + 1] = (int32_t)compact3(k >> 1);
      m.node_xyz[3 * n + 2] = (int32_t)compact3(k >> 2);
    }
  });

  // ---- 3. balance via a dense owner map of the finest cells (the leaves are disjoint, so the
  // threads paint disjoint cells)
  {
    std::vector<int32_t> &owner = m.cellmap;
    owner.assign((size_t)(fx * fy * fz), 0);
    chunked(host_threads(Ne), (size_t)Ne, [&](int, size_t lo, size_t hi) {
      for (size_t e = lo; e < hi; ++e) {
        const int32_t *l = &m.leaf[4 * e];
        const int32_t s = 1 << (L - l[3]);
        for (int z = 0; z < s; ++z)
          for (int y = 0; y < s; ++y) {
            int32_t *row = &owner[((size_t)(l[2] + z) * fy + (l[1] + y)) * fx + l[0]];
            for (int x = 0; x < s; ++x) row[x] = (int32_t)e;
          }
      }
    });
    const int nt = host_threads(Nn);
    std::vector<uint8_t> unbalanced(nt, 0);
    chunked(nt, (size_t)Nn, [&](int t, size_t lo, size_t hi) {
      for (size_t n = lo; n < hi; ++n) {
        const int32_t px = m.node_xyz[3 * n], py = m.node_xyz[3 * n + 1], pz = m.node_xyz[3 * n + 2];
        int lv_lo = 1 << 30, lv_hi = -1;
        for (int c = 0; c < 8; ++c) {
          const int64_t cx = px - 1 + (c & 1), cy = py - 1 + ((c >> 1) & 1), cz = pz - 1 + ((c >> 2) & 1);
          if (cx < 0 || cy < 0 || cz < 0 || cx >= fx || cy >= fy || cz >= fz) continue;
          const int lv = m.leaf[4 * owner[((size_t)cz * fy + cy) * fx + cx] + 3];
          lv_lo = std::min(lv_lo, lv);
          lv_hi = std::max(lv_hi, lv);
        }
        if (lv_hi - lv_lo > 1) {
          unbalanced[t] = 1;
          return;
        }
      }
    });
    for (uint8_t u : unbalanced)
      if (u) return "mesh is not 2:1 balanced";
  }

  // ---- 4. hanging nodes: edge midpoints and face centres that are nodes
  m.hang_index.assign(Nn, -1);
  std::vector<std::array<int32_t, 4>> masters;
  {
    static const int edges[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3},
                                     {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
    static const int faces[6][4] = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5},
                                    {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
    // probes in parallel over element chunks (edge midpoints and face centres that are nodes,
    // with their sorted masters), merged in element order
    struct Found { int32_t n; std::array<int32_t, 4> ms; };
    const int nt = host_threads(Ne);
    std::vector<std::vector<Found>> found(nt);
    // (each thread fills a vector of its own and hands it over at the end: vectors side by side in
    // one array would share the cache lines of their end pointers)
    chunked(nt, (size_t)Ne, [&](int t, size_t lo, size_t hi) {
      std::vector<Found> out;
      for (size_t e = lo; e < hi; ++e) {
        const int32_t *l = &m.leaf[4 * e];
        const int32_t s = 1 << (L - l[3]);
        if (s < 2) continue;
        const int32_t *cn = &m.conn[8 * e];
        auto probe = [&](const int *cs, int nc) {
          int64_t x = 0, y = 0, z = 0;
          for (int i = 0; i < nc; ++i) {
            x += m.node_xyz[3 * cn[cs[i]]];
            y += m.node_xyz[3 * cn[cs[i]] + 1];
            z += m.node_xyz[3 * cn[cs[i]] + 2];
          }
          x /= nc; y /= nc; z /= nc;
          const uint64_t ck = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
          int64_t n;
          if (bm.empty()) {
            n = find_key(m.node_key, ck);
          } else {
            const uint64_t w = ck >> 6, bit = 1ull << (ck & 63);
            n = w < bm.size() && (bm[w] & bit) ? below[w] + __builtin_popcountll(bm[w] & (bit - 1)) : -1;
          }
          if (n < 0) return;
          Found f{(int32_t)n, {-1, -1, -1, -1}};
          for (int i = 0; i < nc; ++i) f.ms[i] = cn[cs[i]];
          std::sort(f.ms.begin(), f.ms.begin() + nc);
          out.push_back(f);
        };
        for (auto &ed : edges) probe(ed, 2);
        for (auto &fc : faces) probe(fc, 4);
      }
      found[t].swap(out);
    });
    for (const auto &fv : found)
      for (const Found &f : fv) {
        if (m.hang_index[f.n] < 0) {
          m.hang_index[f.n] = (int32_t)masters.size();
          masters.push_back(f.ms);
          m.hang_node.push_back(f.n);
        } else if (masters[m.hang_index[f.n]] != f.ms) {
          return "inconsistent hanging-node constraints";
        }
      }
    // ascending node order
    std::vector<int32_t> ord(m.hang_node.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return m.hang_node[a] < m.hang_node[b]; });
    std::vector<int32_t> hn(ord.size());
    m.hang_master.resize(4 * ord.size());
    for (size_t i = 0; i < ord.size(); ++i) {
      hn[i] = m.hang_node[ord[i]];
      for (int j = 0; j < 4; ++j) m.hang_master[4 * i + j] = masters[ord[i]][j];
      m.hang_index[hn[i]] = (int32_t)i;
    }
    m.hang_node.swap(hn);
    for (size_t i = 0; i < m.hang_node.size(); ++i)
      for (int j = 0; j < 4; ++j) {
        const int32_t mm = m.hang_master[4 * i + j];
        if (mm >= 0 && m.hang_index[mm] >= 0) return "constraint chain (master is hanging)";
      }
  }

  std::vector<uint64_t>().swap(bm);
  std::vector<int64_t>().swap(below);

  // ---- 5. flags
  m.nflag.assign(Nn, 0);
  const int64_t ext[3] = {fx, fy, fz};
  for (int64_t n = 0; n < Nn; ++n) {
    for (int f = 0; f < 6; ++f)
      if ((d.dirichlet_faces >> f) & 1) {
        const int a = f / 2, side = f % 2;
        if (m.node_xyz[3 * n + a] == (side ? ext[a] : 0)) m.nflag[n] |= 1;
      }
    if (m.hang_index[n] >= 0) m.nflag[n] |= 2;
    if (m.nflag[n] & 1) m.n_dirichlet++;
    if (!m.nflag[n]) m.n_free_nodes++;
  }

  m.K0.resize(576);
  reference_stiffness(d.nu, m.K0.data());
  {
    // K0 in the butterfly basis: K0m = T K0 T^T / 64 with T[(m,c)][(k,c)] = prod over axes a
    // with bit a of m set of (bit a of k ? +1 : -1).  Check that it is block diagonal over
    // signatures (DOF c of block s = mode s ^ (1 << c)) and keep the 8 blocks.
    auto t8 = [](int mm, int k) {
      int v = 1;
      for (int a = 0; a < 3; ++a)
        if ((mm >> a) & 1) v *= ((k >> a) & 1) ? 1 : -1;
      return v;
    };
    double Km[24][24] = {};
    double mx = 0;
    for (int r = 0; r < 24; ++r)
      for (int q = 0; q < 24; ++q) {
        const int mr = r / 3, cr = r % 3, mq = q / 3, cq = q % 3;
        double acc = 0;
        for (int k = 0; k < 8; ++k)
          for (int l = 0; l < 8; ++l) acc += t8(mr, k) * m.K0[(3 * k + cr) * 24 + 3 * l + cq] * t8(mq, l);
        Km[r][q] = acc / 64.0;
        mx = std::max(mx, std::fabs(Km[r][q]));
      }
    auto sig = [](int mm, int c) { return mm ^ (1 << c); };
    for (int r = 0; r < 24; ++r)
      for (int q = 0; q < 24; ++q)
        if (sig(r / 3, r % 3) != sig(q / 3, q % 3) && std::fabs(Km[r][q]) > 1e-13 * mx)
          return "element matrix is not block diagonal in the butterfly basis";
    m.modal.assign(72, 0.0);
    for (int sgn = 0; sgn < 8; ++sgn)
      for (int c = 0; c < 3; ++c)
        for (int c2 = 0; c2 < 3; ++c2) {
          const int r = 3 * (sgn ^ (1 << c)) + c, q = 3 * (sgn ^ (1 << c2)) + c2;
          double v = Km[r][q];
          if (std::fabs(v) <= 1e-13 * mx) v = 0.0;
          m.modal[sgn * 9 + c * 3 + c2] = v;
        }
    // rows and columns of the rigid translations vanish
    for (int c = 0; c < 3; ++c)
      for (int c2 = 0; c2 < 3; ++c2) {
        const int sgn = 1 << c;
        if (m.modal[sgn * 9 + c * 3 + c2] != 0.0 || m.modal[sgn * 9 + c2 * 3 + c] != 0.0)
          return "translation modes are not in the null space of the element matrix";
      }
  }

  // ---- 6. operator blocks: chunks of consecutive elements, local nodes, colours
  // Local nodes of a block: its regular ("effective") nodes -- regular corners
  // and masters of hanging corners -- shared ones first, then the hanging
  // corners it uses.  Elements address corners by local id; the hanging slots
  // are filled from their masters before the element pass and folded back into
  // them after it.
  std::vector<int32_t> nblocks_of(Nn, 0);       // number of blocks and bricks touching a regular node
  // ---- 6a. bricks: aligned 4x4x4 cubes of 64 equal-level elements (consecutive in the Morton
  // order, element t of the brick at (i, j, k) with t = morton(i, j, k)) whose hanging corners --
  // on faces and edges shared with coarser elements -- each have their masters at the lattice
  // nodes next to them along the coarse edge or face.  The brick's nodes form a 5x5x5 lattice,
  // node (a, b, c) at a + 5 b + 25 c; the brick pass addresses them implicitly.  Other elements
  // form the blocks.
  std::vector<uint8_t> in_brick(Ne, 0);
  m.brick_e0.clear();
  m.brick_node.clear();
  m.brick_hax.clear();
  m.brick_fold.clear();
  {
    auto demorton = [](int t, int &i, int &j, int &k) {
      i = (t & 1) | ((t >> 2) & 2);
      j = ((t >> 1) & 1) | ((t >> 3) & 2);
      k = ((t >> 2) & 1) | ((t >> 4) & 2);
    };
    auto morton6 = [](int i, int j, int k) {
      return (i & 1) | ((j & 1) << 1) | ((k & 1) << 2) | ((i & 2) << 2) | ((j & 2) << 3) | ((k & 2) << 4);
    };
    // Whether element e starts a brick depends only on the elements and nodes around it (two
    // aligned cubes of equal-level elements never overlap unless they coincide), so the starts
    // are found in parallel over element chunks, each chunk's bricks in element order.
    struct Found {
      int64_t e;
      int32_t lat[125];
      uint8_t hax[125];
      uint32_t fold[125];
    };
    auto check = [&](int64_t e, Found &f) -> bool {
      int32_t *lat = f.lat;
      uint8_t *hax = f.hax;
      const int32_t *l0 = &m.leaf[4 * e];
      const int32_t s = 1 << (L - l0[3]);
      bool ok = l0[0] % (4 * s) == 0 && l0[1] % (4 * s) == 0 && l0[2] % (4 * s) == 0;
      for (int t = 1; ok && t < 64; ++t) {
        int i, j, k;
        demorton(t, i, j, k);
        const int32_t *lt = &m.leaf[4 * (e + t)];
        ok = lt[3] == l0[3] && lt[0] == l0[0] + s * i && lt[1] == l0[1] + s * j && lt[2] == l0[2] + s * k;
      }
      if (!ok) return false;
      for (int c = 0; c < 5; ++c)
        for (int b = 0; b < 5; ++b)
          for (int a = 0; a < 5; ++a) {
            const int ex = a < 4 ? a : 3, ey = b < 4 ? b : 3, ez = c < 4 ? c : 3;
            const int q = (a - ex) + 2 * (b - ey) + 4 * (c - ez);
            lat[a + 5 * b + 25 * c] = m.conn[8 * (e + morton6(ex, ey, ez)) + q];
          }
      for (int nd = 0; nd < 125; ++nd) {
        hax[nd] = 0;
        const int32_t hi = m.hang_index[lat[nd]];
        if (hi < 0) continue;
        const int a = nd % 5, b = (nd / 5) % 5, c = nd / 25;
        int nm = 0, dmask = 0;
        int step[4][3];
        for (int q = 0; q < 4; ++q) {
          const int32_t mm = m.hang_master[4 * hi + q];
          if (mm < 0) continue;
          const int32_t *p = &m.node_xyz[3 * mm];
          const int32_t rel[3] = {p[0] - l0[0] - s * a, p[1] - l0[1] - s * b, p[2] - l0[2] - s * c};
          for (int ax = 0; ax < 3; ++ax) {
            if (rel[ax] != 0 && rel[ax] != s && rel[ax] != -s) return false;
            step[nm][ax] = rel[ax] / s;
            if (rel[ax] != 0) dmask |= 1 << ax;
          }
          if (m.hang_index[mm] >= 0) return false;
          ++nm;
        }
        const int naxes = (dmask & 1) + ((dmask >> 1) & 1) + ((dmask >> 2) & 1);
        if (!((nm == 2 && naxes == 1) || (nm == 4 && naxes == 2))) return false;
        // every master moves by exactly one lattice step along each interpolation axis, and
        // the masters are distinct
        for (int q = 0; q < nm; ++q)
          for (int ax = 0; ax < 3; ++ax)
            if (((dmask >> ax) & 1) ? (step[q][ax] == 0) : (step[q][ax] != 0)) return false;
        for (int q = 0; q < nm; ++q)
          for (int r = q + 1; r < nm; ++r)
            if (step[q][0] == step[r][0] && step[q][1] == step[r][1] && step[q][2] == step[r][2]) return false;
        for (int ax = 0; ax < 3; ++ax) {
          const int pos = ax == 0 ? a : (ax == 1 ? b : c);
          if (((dmask >> ax) & 1) && (pos == 0 || pos == 4)) return false;
        }
        hax[nd] = (uint8_t)dmask;
      }
      // fold masks: which lattice neighbours of a regular node are hanging nodes it is a master
      // of -- bits 2 ax + (step > 0): the neighbour one step along axis ax, edge-hanging along
      // ax; bits 6 + 4 pl + 2 (step1 > 0) + (step0 > 0): the diagonal neighbour in coordinate
      // plane pl ((x, y), (x, z), (y, z)), face-hanging in that plane
      for (int nd = 0; nd < 125; ++nd) {
        uint32_t fm = 0;
        const int pos[3] = {nd % 5, (nd / 5) % 5, nd / 25}, nst[3] = {1, 5, 25};
        if (!hax[nd]) {
          for (int ax = 0; ax < 3; ++ax)
            for (int sg = -1; sg <= 1; sg += 2) {
              const int p = pos[ax] + sg;
              if (p >= 0 && p <= 4 && hax[nd + sg * nst[ax]] == (1 << ax)) fm |= 1u << (2 * ax + (sg > 0));
            }
          for (int pl = 0; pl < 3; ++pl) {
            const int ax0 = pl == 2 ? 1 : 0, ax1 = pl == 0 ? 1 : 2;
            for (int s1g = -1; s1g <= 1; s1g += 2)
              for (int s0g = -1; s0g <= 1; s0g += 2) {
                const int p0 = pos[ax0] + s0g, p1 = pos[ax1] + s1g;
                if (p0 < 0 || p0 > 4 || p1 < 0 || p1 > 4) continue;
                if (hax[nd + s0g * nst[ax0] + s1g * nst[ax1]] == ((1 << ax0) | (1 << ax1)))
                  fm |= 1u << (6 + 4 * pl + 2 * (s1g > 0) + (s0g > 0));
              }
          }
        }
        f.fold[nd] = fm;
      }
      return true;
    };
    const int64_t ncand = Ne >= 64 ? Ne - 63 : 0;
    const int nt = host_threads(ncand);
    std::vector<std::vector<Found>> found(nt);
    chunked(nt, (size_t)ncand, [&](int t, size_t lo, size_t hi) {
      std::vector<Found> out;
      Found f;
      for (size_t e = lo; e < hi; ++e)
        if (check((int64_t)e, f)) {
          f.e = (int64_t)e;
          out.push_back(f);
        }
      found[t].swap(out);
    });
    for (const auto &fv : found)
      for (const Found &f : fv) {
        m.brick_e0.push_back((int32_t)f.e);
        m.brick_fold.insert(m.brick_fold.end(), f.fold, f.fold + 125);
        for (int nd = 0; nd < 125; ++nd) {
          uint32_t g = (uint32_t)f.lat[nd];
          if (m.nflag[f.lat[nd]] & 1) g |= 0x80000000u;
          m.brick_node.push_back((int32_t)g);
          m.brick_hax.push_back(f.hax[nd]);
          if (!f.hax[nd]) nblocks_of[f.lat[nd]]++;
        }
        std::memset(&in_brick[f.e], 1, 64);
      }
    m.nbrick = (int32_t)m.brick_e0.size();
  }
  // blocks: consecutive runs of the non-brick elements in Morton order (gen), at most kBlockElems
  // elements and kMaxLocal local nodes each; a block may span the bricks between its elements
  std::vector<int32_t> &gen = m.gen_elem;
  gen.clear();
  for (int64_t e = 0; e < Ne; ++e)
    if (!in_brick[e]) gen.push_back((int32_t)e);
  const int64_t ngen = (int64_t)gen.size();
  struct Blk { int64_t e0, e1; };   // range of gen
  std::vector<Blk> blks;
  {
    std::vector<int32_t> mark(Nn, -1);
    auto count_local = [&](int64_t u0, int64_t u1, int tag) {
      int cnt = 0;
      for (int64_t u = u0; u < u1; ++u)
        for (int k = 0; k < 8; ++k) {
          const int64_t e = gen[u];
          const int32_t n = m.conn[8 * e + k];
          if (mark[n] != tag) { mark[n] = tag; ++cnt; }
          const int32_t h = m.hang_index[n];
          if (h >= 0)
            for (int j = 0; j < 4; ++j) {
              const int32_t mm = m.hang_master[4 * h + j];
              if (mm >= 0 && mark[mm] != tag) { mark[mm] = tag; ++cnt; }
            }
        }
      return cnt;
    };
    int tag = 0;
    int64_t u0 = 0;
    while (u0 < ngen) {
      int64_t len = std::min<int64_t>(kBlockElems, ngen - u0);
      while (len > 1 && count_local(u0, u0 + len, tag++) > kMaxLocal) len = (len + 1) / 2;
      if (count_local(u0, u0 + len, tag++) > kMaxLocal) return "block local-node limit exceeded";
      blks.push_back({u0, u0 + len});
      u0 += len;
    }
  }
  const int32_t nblk = (int32_t)blks.size();
  m.nblk = nblk;
  // Every block's lists depend on its own elements and on nblocks_of alone, so contiguous ranges of
  // blocks are built on host threads, each with a node -> local id map of its own (capped so the
  // maps stay within 512 MB), and concatenated in block order with the running offsets of a
  // sequential pass.
  const int nbt = std::max(1, std::min(host_threads((size_t)nblk * 4096), (int)((int64_t(1) << 27) / std::max<int64_t>(Nn, 1))));
  std::vector<std::vector<int32_t>> bl(nblk);   // regular nodes per block, ascending
  chunked(nbt, (size_t)nblk, [&](int, size_t lo, size_t hi) {
    for (size_t b = lo; b < hi; ++b) {
      std::vector<int32_t> v;
      for (int64_t u = blks[b].e0; u < blks[b].e1; ++u)
        for (int k = 0; k < 8; ++k) {
          const int32_t n = m.conn[8 * (int64_t)gen[u] + k];
          const int32_t h = m.hang_index[n];
          if (h < 0) v.push_back(n);
          else
            for (int j = 0; j < 4; ++j)
              if (m.hang_master[4 * h + j] >= 0) v.push_back(m.hang_master[4 * h + j]);
        }
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
      for (int32_t n : v) __atomic_fetch_add(&nblocks_of[n], 1, __ATOMIC_RELAXED);
      bl[b].swap(v);
    }
  });
  m.blk_elem.assign(2 * (size_t)nblk, 0);
  m.blk_node.assign(nblk + 1, 0);
  m.blk_shared.assign(nblk, 0);
  m.blk_slot.assign(nblk + 1, 0);
  m.blk_hang.assign(nblk + 1, 0);
  m.blk_iptr.assign(nblk + 1, 0);
  m.blk_inv.assign(nblk, 0);
  m.lcorner.assign(8 * (size_t)Ne, 0);
  // per block: nreg, nshared, nhang, ninv (its lists' lengths); per thread: the lists
  std::vector<std::array<int32_t, 4>> bsz(nblk);
  struct BlkLists { std::vector<int32_t> lnode; std::vector<uint16_t> hent, iptr, inv; };
  std::vector<BlkLists> bls(nbt);
  std::vector<const char *> berr(nbt, nullptr);
  std::vector<int32_t> bmax(nbt, 0);
  chunked(nbt, (size_t)nblk, [&](int t, size_t lo, size_t hi) {
    BlkLists out;
    std::vector<int32_t> local_of(Nn, -1);
    std::vector<int32_t> lcount, lfill;          // per-block CSR scratch of the inverse lists
    int32_t max_local = 0;
    for (size_t b = lo; b < hi; ++b) {
      const std::vector<int32_t> &v = bl[b];
      std::vector<int32_t> order;
      order.reserve(v.size());
      for (int32_t n : v) if (nblocks_of[n] > 1) order.push_back(n);
      const int32_t nshared = (int32_t)order.size();
      for (int32_t n : v) if (nblocks_of[n] == 1) order.push_back(n);
      const int32_t nreg = (int32_t)order.size();
      for (int32_t i = 0; i < nreg; ++i) local_of[order[i]] = i;
      out.lnode.insert(out.lnode.end(), order.begin(), order.end());
      // hanging nodes used by this block: local ids nreg, nreg+1, ... in first-use order
      std::vector<int32_t> used_h;
      const int64_t e0 = blks[b].e0, e1 = blks[b].e1;   // range of gen
      for (int64_t u = e0; u < e1; ++u)
        for (int k = 0; k < 8; ++k) {
          const int32_t n = m.conn[8 * (int64_t)gen[u] + k];
          if (m.hang_index[n] >= 0 && local_of[n] < 0) {
            local_of[n] = nreg + (int32_t)used_h.size();
            used_h.push_back(m.hang_index[n]);
          }
        }
      const int32_t nloc = nreg + (int32_t)used_h.size();
      if (nloc > kMaxLocal) { berr[t] = "block local-node limit exceeded"; break; }
      max_local = std::max(max_local, nloc);
      for (int64_t u = e0; u < e1; ++u)
        for (int k = 0; k < 8; ++k) {
          const int64_t e = gen[u];
          m.lcorner[8 * e + k] = (uint16_t)local_of[m.conn[8 * e + k]];
        }
      // inverse lists, built as one block-local CSR: per local node its slots (element order),
      // then its fold entries (hanging order)
      if (used_h.size() >= (size_t)kQuarterBit) { berr[t] = "too many hanging nodes in a block"; break; }
      lcount.assign(nloc + 1, 0);
      for (int64_t u = e0; u < e1; ++u)
        for (int k = 0; k < 8; ++k) lcount[local_of[m.conn[8 * (int64_t)gen[u] + k]] + 1]++;
      for (size_t j = 0; j < used_h.size(); ++j)
        for (int q = 0; q < 4; ++q) {
          const int32_t mm = m.hang_master[4 * used_h[j] + q];
          if (mm >= 0) lcount[local_of[mm] + 1]++;
        }
      for (int32_t i = 0; i < nloc; ++i) lcount[i + 1] += lcount[i];
      if (lcount[nloc] > 0xFFFF) { berr[t] = "inverse list of a block too long"; break; }
      const size_t inv0 = out.inv.size();
      out.inv.resize(inv0 + lcount[nloc]);
      lfill.assign(lcount.begin(), lcount.end() - 1);
      for (int64_t u = e0; u < e1; ++u)
        for (int k = 0; k < 8; ++k)   // the slot's offset in the block's per-element result buffer
          out.inv[inv0 + lfill[local_of[m.conn[8 * (int64_t)gen[u] + k]]]++] = (uint16_t)((u - e0) * kSlotRow + 3 * k);
      for (size_t j = 0; j < used_h.size(); ++j) {
        const int32_t h = used_h[j];
        const bool quarter = m.hang_master[4 * h + 2] >= 0;
        for (int q = 0; q < 4; ++q) {
          const int32_t mm = m.hang_master[4 * h + q];
          out.hent.push_back(mm >= 0 ? (uint16_t)local_of[mm] : (uint16_t)0xFFFF);
          if (mm >= 0)
            out.inv[inv0 + lfill[local_of[mm]]++] = (uint16_t)(kFoldBit | (quarter ? kQuarterBit : 0) | j);
        }
      }
      for (int32_t i = 0; i <= nloc; ++i) out.iptr.push_back((uint16_t)lcount[i]);
      bsz[b] = {nreg, nshared, (int32_t)used_h.size(), lcount[nloc]};
      m.blk_elem[2 * b] = (int32_t)e0;
      m.blk_elem[2 * b + 1] = (int32_t)e1;
      for (int32_t n : order) local_of[n] = -1;
      for (int32_t h : used_h) local_of[m.hang_node[h]] = -1;
    }
    bmax[t] = max_local;
    bls[t] = std::move(out);
  });
  for (int t = 0; t < nbt; ++t)
    if (berr[t]) return berr[t];
  int32_t max_local = 0;
  for (int t = 0; t < nbt; ++t) max_local = std::max(max_local, bmax[t]);
  {
    // running offsets in 64 bits: the tables keep them in 32
    int64_t node = 0, slot = 0, hang = 0, iptr = 0, inv = 0;
    for (int32_t b = 0; b < nblk; ++b) {
      const int32_t nreg = bsz[b][0], nshared = bsz[b][1], nhang = bsz[b][2], nloc = nreg + nhang;
      m.blk_shared[b] = nshared;
      m.blk_inv[b] = (int32_t)inv;
      node += nreg;
      slot += nshared;
      hang += nhang;
      iptr += nloc + 1;
      inv += bsz[b][3];
      if (std::max({node, slot, 4 * hang, iptr, inv}) > kMaxOffset) return kTooLarge;
      m.blk_node[b + 1] = (int32_t)node;
      m.blk_slot[b + 1] = (int32_t)slot;
      m.blk_hang[b + 1] = (int32_t)hang;
      m.blk_iptr[b + 1] = (int32_t)iptr;
    }
  }
  for (int t = 0; t < nbt; ++t) {
    m.lnode.insert(m.lnode.end(), bls[t].lnode.begin(), bls[t].lnode.end());
    m.hent.insert(m.hent.end(), bls[t].hent.begin(), bls[t].hent.end());
    m.iptr.insert(m.iptr.end(), bls[t].iptr.begin(), bls[t].iptr.end());
    m.inv.insert(m.inv.end(), bls[t].inv.begin(), bls[t].inv.end());
    bls[t] = BlkLists();
  }
  m.max_local = max_local;

  // ---- 7. second pass over shared nodes: the partials of a shared node are
  // contiguous (node-major CSR, ascending block order inside a node), so the
  // second pass streams them; each block writes its shared nodes' partials to
  // their CSR positions (lslot).
  {
    // blocks first (ascending), then bricks (ascending): the order of a node's partials.  The
    // units (blocks, then bricks) are split into chunks; each chunk counts its partials per node,
    // then writes them after the earlier chunks' partials of the same node, which is the order
    // of one pass over the units (the threads' counts take nt x Nn int32: capped at 512 MB).
    const int64_t nunit = (int64_t)nblk + m.nbrick;
    const int nt = std::max(1, std::min(host_threads((size_t)nunit * 512),
                                        (int)(((int64_t)1 << 27) / std::max<int64_t>(Nn, 1))));
    auto unit_partials = [&](size_t lo, size_t hi, auto &&emit) {
      for (size_t u = lo; u < hi; ++u) {
        if ((int64_t)u < nblk) {
          const int32_t b = (int32_t)u;
          for (int32_t i = 0; i < m.blk_shared[b]; ++i) emit(m.lnode[m.blk_node[b] + i], &m.lslot[m.blk_slot[b] + i]);
        } else {
          const size_t i0 = (size_t)125 * (u - nblk);
          for (size_t i = i0; i < i0 + 125; ++i) {
            const int32_t n = m.brick_node[i] & 0x7FFFFFFF;
            if (m.brick_hax[i]) m.brick_out[i] = -2;
            else if (nblocks_of[n] > 1) emit(n, &m.brick_out[i]);
          }
        }
      }
    };
    m.lslot.assign(m.blk_slot[nblk], 0);
    m.brick_out.assign(m.brick_node.size(), -1);
    std::vector<int32_t> ccnt((size_t)nt * Nn, 0);
    chunked(nt, (size_t)nunit, [&](int t, size_t lo, size_t hi) {
      int32_t *c = &ccnt[(size_t)t * Nn];
      unit_partials(lo, hi, [&](int32_t n, int32_t *) { c[n]++; });
    });
    std::vector<int32_t> start(Nn + 1, 0);
    chunked(host_threads(Nn), (size_t)Nn, [&](int, size_t lo, size_t hi) {
      for (size_t n = lo; n < hi; ++n) {
        int32_t v = 0;
        for (int t = 0; t < nt; ++t) v += ccnt[(size_t)t * Nn + n];
        start[n + 1] = v;
      }
    });
    // shared nodes: those with partials, ascending
    std::vector<uint8_t> has(Nn);
    for (int64_t n = 0; n < Nn; ++n) has[n] = start[n + 1] > 0;
    {
      int64_t run = 0;
      for (int64_t n = 0; n < Nn; ++n) {
        run += start[n + 1];
        if (3 * run > kMaxOffset) return kTooLarge;   // 3 partials per shared slot
        start[n + 1] = (int32_t)run;
      }
    }
    chunked(host_threads(Nn), (size_t)Nn, [&](int, size_t lo, size_t hi) {
      for (size_t n = lo; n < hi; ++n) {
        int32_t s0 = start[n];
        for (int t = 0; t < nt; ++t) {
          const int32_t v = ccnt[(size_t)t * Nn + n];
          ccnt[(size_t)t * Nn + n] = s0;
          s0 += v;
        }
      }
    });
    chunked(nt, (size_t)nunit, [&](int t, size_t lo, size_t hi) {
      int32_t *f = &ccnt[(size_t)t * Nn];
      unit_partials(lo, hi, [&](int32_t n, int32_t *slot) { *slot = f[n]++; });
    });
    m.nslot = start[Nn];
    // the brick pass's packed table: per brick 3 x 128 int32 -- node ids (125, then e0 at 125),
    // output targets (125), fold mask | axes << 24 (125)
    m.brick_tab.assign((size_t)384 * m.nbrick, 0);
    chunked(host_threads((size_t)m.nbrick * 128), (size_t)m.nbrick, [&](int, size_t lo, size_t hi) {
      for (size_t bk = lo; bk < hi; ++bk) {
        int32_t *t = &m.brick_tab[(size_t)384 * bk];
        for (int nd = 0; nd < 125; ++nd) {
          const size_t i = (size_t)125 * bk + nd;
          t[nd] = m.brick_node[i];
          t[128 + nd] = m.brick_out[i];
          t[256 + nd] = (int32_t)(m.brick_fold[i] | ((uint32_t)m.brick_hax[i] << 24));
        }
        t[125] = m.brick_e0[bk];
      }
    });
    m.sh_ptr.push_back(0);
    m.sh_of_node.assign(Nn, -1);
    for (int64_t n = 0; n < Nn; ++n)
      if (has[n]) {
        m.sh_of_node[n] = (int32_t)m.sh_node.size();
        m.sh_node.push_back((int32_t)n);
        m.sh_ptr.push_back(start[n + 1]);
      }
  }

  // ---- 7b. one contiguous record per block (16-byte aligned), staged into
  // shared memory by the operator kernel with coalesced 16-byte loads:
  //   header (16 x i32: first element, ne, nreg, nshared, nhang, ninv, byte offsets of
  //   lslot, hent, iptr, inv, lcorner, lnode, elist, 3 x 0), lcorner (8 x u16 per element: the
  //   local ids of its corners), lnode (i32, bit 31 = Dirichlet node), lslot
  //   (i32), hent (4 x u16), iptr (u16), inv (u16); elist (i32 per element: its canonical index)
  //   follows lcorner.
  {
    m.rec_off.assign(nblk + 1, 0);
    m.rec_skip.assign(nblk, 0);
    m.max_rec_bytes = 0;
    m.max_rec_stage = 0;
    auto align = [](size_t v, size_t a) { return (v + a - 1) / a * a; };
    struct Layout { int32_t nreg, nshared, nhang, nloc, ninv, ne; size_t o_lcorner, o_elist, o_lnode, o_lslot, o_hent, o_iptr, o_inv, bytes; };
    auto layout = [&](int32_t b) {
      Layout y;
      y.nreg = m.blk_node[b + 1] - m.blk_node[b];
      y.nshared = m.blk_shared[b];
      y.nhang = m.blk_hang[b + 1] - m.blk_hang[b];
      y.nloc = y.nreg + y.nhang;
      y.ninv = m.iptr[m.blk_iptr[b] + y.nloc];
      y.ne = m.blk_elem[2 * b + 1] - m.blk_elem[2 * b];
      size_t off = 64;
      y.o_lcorner = off; off += 16 * (size_t)y.ne;
      y.o_elist = off; off += 4 * (size_t)y.ne;
      off = align(off, 16);   // the sections from lnode on are staged into shared memory
      y.o_lnode = off; off += 4 * (size_t)y.nreg;
      y.o_lslot = off; off += 4 * (size_t)y.nshared;
      off = align(off, 8);
      y.o_hent = off; off += 8 * (size_t)y.nhang;
      y.o_iptr = off; off += 2 * (size_t)(y.nloc + 1);
      y.o_inv = off; off += 2 * (size_t)y.ninv;
      y.bytes = align(off, 16);
      return y;
    };
    // the offsets in block order, then the records written in parallel
    int64_t rec_units = 0;
    for (int32_t b = 0; b < nblk; ++b) {
      const Layout y = layout(b);
      rec_units += (int64_t)(y.bytes / 16);
      if (rec_units > kMaxOffset) return kTooLarge;
      m.rec_off[b + 1] = (int32_t)rec_units;
      m.max_rec_bytes = std::max<int32_t>(m.max_rec_bytes, (int32_t)y.bytes);
      m.rec_skip[b] = (int32_t)((y.o_lnode - 64) / 16);
      m.max_rec_stage = std::max<int32_t>(m.max_rec_stage, (int32_t)(y.bytes - (y.o_lnode - 64)));
    }
    m.brec.assign(16 * (size_t)m.rec_off[nblk], 0);
    chunked(host_threads((size_t)nblk * 4096), (size_t)nblk, [&](int, size_t lo, size_t hi) {
      for (size_t b = lo; b < hi; ++b) {
        const Layout y = layout((int32_t)b);
        uint8_t *rec = &m.brec[16 * (size_t)m.rec_off[b]];
        const int32_t *el = &gen[m.blk_elem[2 * b]];
        int32_t hdr[16] = {el[0], y.ne, y.nreg, y.nshared, y.nhang, y.ninv, (int32_t)y.o_lslot, (int32_t)y.o_hent,
                           (int32_t)y.o_iptr, (int32_t)y.o_inv, (int32_t)y.o_lcorner, (int32_t)y.o_lnode,
                           (int32_t)y.o_elist, 0, 0, 0};
        std::memcpy(rec, hdr, sizeof(hdr));
        for (int32_t t = 0; t < y.ne; ++t) std::memcpy(&rec[y.o_lcorner + 16 * (size_t)t], &m.lcorner[8 * (size_t)el[t]], 16);
        std::memcpy(&rec[y.o_elist], el, 4 * (size_t)y.ne);
        for (int32_t i = 0; i < y.nreg; ++i) {
          uint32_t g = (uint32_t)m.lnode[m.blk_node[b] + i];
          if (m.nflag[g] & 1) g |= 0x80000000u;
          std::memcpy(&rec[y.o_lnode + 4 * i], &g, 4);
        }
        if (y.nshared) std::memcpy(&rec[y.o_lslot], &m.lslot[m.blk_slot[b]], 4 * (size_t)y.nshared);
        if (y.nhang) std::memcpy(&rec[y.o_hent], &m.hent[4 * (size_t)m.blk_hang[b]], 8 * (size_t)y.nhang);
        std::memcpy(&rec[y.o_iptr], &m.iptr[m.blk_iptr[b]], 2 * (size_t)(y.nloc + 1));
        if (y.ninv) std::memcpy(&rec[y.o_inv], &m.inv[m.blk_inv[b]], 2 * (size_t)y.ninv);
      }
    });
  }

  // ---- 8. Jacobi diagonal coefficients: d_{m,c} = sum_e c_e q_{e,m,c}
  {
    // coefficient triples by their bit patterns; the maps only number them in order of first
    // appearance, so their iteration order never matters
    struct TripleHash {
      size_t operator()(const std::array<int64_t, 3> &k) const {
        uint64_t h = 0x9E3779B97F4A7C15ull;
        for (int c = 0; c < 3; ++c) h = (h ^ (uint64_t)k[c]) * 0xFF51AFD7ED558CCDull;
        return (size_t)(h ^ (h >> 29));
      }
    };
    using TripleMap = std::unordered_map<std::array<int64_t, 3>, int, TripleHash>;
    TripleMap tab_index;
    {
      // entry 0: a corner that is its own node in an element without hanging corners
      const double q = m.K0[0];
      std::array<int64_t, 3> kq;
      for (int c = 0; c < 3; ++c) std::memcpy(&kq[c], &q, 8);
      tab_index[kq] = 0;
      m.dg_tab.insert(m.dg_tab.end(), {q, q, q});
    }
    // pass 1 (in parallel over element chunks): elements with hanging corners list their
    // (node, coefficient triple) entries in element order; every chunk numbers the distinct
    // triples it meets in order of first appearance, and the chunks' numberings are merged in
    // chunk order, so the table is the one an element-order pass would build
    // (the threads' node counts below take nt x Nn int32: capped at 512 MB)
    const int nt = std::max(1, std::min(host_threads(Ne), (int)((int64_t(1) << 27) / std::max<int64_t>(Nn, 1))));
    std::vector<std::vector<int32_t>> cx_node(nt), cx_lq(nt);
    std::vector<std::vector<std::array<double, 3>>> cx_tab(nt);
    std::vector<int32_t> ex_end(Ne, 0);   // per element: end of its entries within its chunk's list
    std::vector<uint8_t> plain(Ne);       // per element: no hanging corners
    chunked(nt, (size_t)Ne, [&](int t, size_t lo, size_t hi) {
      TripleMap local;
      std::vector<int32_t> my_node, my_lq;   // handed over at the end (no shared cache lines)
      std::vector<std::array<double, 3>> my_tab;
      for (size_t e = lo; e < hi; ++e) {
        bool pl = true;
        for (int k = 0; k < 8; ++k) pl &= m.hang_index[m.conn[8 * e + k]] < 0;
        plain[e] = pl;
        if (pl) {
          ex_end[e] = (int32_t)my_node.size();
          continue;
        }
        // corner expansion: (node, weight) pairs
        int32_t nodes[32];
        double wts[32];
        int corner_of[32];
        int np = 0;
        for (int k = 0; k < 8; ++k) {
          const int32_t n = m.conn[8 * e + k];
          const int32_t h = m.hang_index[n];
          if (h < 0) {
            nodes[np] = n; wts[np] = 1.0; corner_of[np++] = k;
          } else {
            int nm = 0;
            for (int j = 0; j < 4; ++j) nm += m.hang_master[4 * h + j] >= 0;
            for (int j = 0; j < nm; ++j) {
              nodes[np] = m.hang_master[4 * h + j]; wts[np] = 1.0 / nm; corner_of[np++] = k;
            }
          }
        }
        int32_t uniq[32];
        int nu_ = 0;
        for (int i = 0; i < np; ++i) {
          bool seen = false;
          for (int j = 0; j < nu_; ++j) seen |= uniq[j] == nodes[i];
          if (!seen) uniq[nu_++] = nodes[i];
        }
        for (int u = 0; u < nu_; ++u) {
          double v[8] = {};
          for (int i = 0; i < np; ++i)
            if (nodes[i] == uniq[u]) v[corner_of[i]] += wts[i];
          // q_c = v^T K0_cc v over the corners where v is nonzero, in ascending corner order
          // (the zero terms of the full double sum add nothing)
          int nz[8], nnz = 0;
          for (int a = 0; a < 8; ++a)
            if (v[a] != 0.0) nz[nnz++] = a;
          std::array<double, 3> q;
          for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int ia = 0; ia < nnz; ++ia)
              for (int ib = 0; ib < nnz; ++ib) {
                const int a = nz[ia], b2 = nz[ib];
                s += v[a] * v[b2] * m.K0[(3 * a + c) * 24 + 3 * b2 + c];
              }
            q[c] = s;
          }
          std::array<int64_t, 3> kq;
          for (int c = 0; c < 3; ++c) std::memcpy(&kq[c], &q[c], 8);
          auto it = local.find(kq);
          int li;
          if (it == local.end()) {
            li = (int)my_tab.size();
            local[kq] = li;
            my_tab.push_back(q);
          } else {
            li = it->second;
          }
          my_node.push_back(uniq[u]);
          my_lq.push_back(li);
        }
        ex_end[e] = (int32_t)my_node.size();
      }
      cx_node[t].swap(my_node);
      cx_lq[t].swap(my_lq);
      cx_tab[t].swap(my_tab);
    });
    for (int t = 0; t < nt; ++t)   // ex_end holds positions in a chunk's list as int32
      if ((int64_t)cx_node[t].size() > kMaxOffset) return kTooLarge;
    std::vector<std::vector<uint16_t>> l2g(nt);
    for (int t = 0; t < nt; ++t)
      for (const auto &q : cx_tab[t]) {
        std::array<int64_t, 3> kq;
        for (int c = 0; c < 3; ++c) std::memcpy(&kq[c], &q[c], 8);
        auto it = tab_index.find(kq);
        int qi;
        if (it == tab_index.end()) {
          qi = (int)tab_index.size();
          if (qi >= 65535) return "too many distinct diagonal coefficients";
          tab_index[kq] = qi;
          m.dg_tab.insert(m.dg_tab.end(), q.begin(), q.end());
        } else {
          qi = it->second;
        }
        l2g[t].push_back((uint16_t)qi);
      }
    // the count of every node per chunk, then each chunk's write position inside every node's
    // list (after the earlier chunks' entries), so the chunks fill the node-major CSR in
    // parallel in element order
    std::vector<int32_t> ccnt((size_t)nt * Nn, 0);
    auto chunk_entries = [&](int t, size_t lo, size_t hi, auto &&emit) {
      int32_t x0 = 0;   // ex_end is relative to the chunk's own list
      for (size_t e = lo; e < hi; ++e) {
        if (plain[e]) {
          for (int k = 0; k < 8; ++k) emit(m.conn[8 * e + k], (int32_t)e, (uint16_t)0);
          continue;
        }
        for (int32_t i = x0; i < ex_end[e]; ++i) emit(cx_node[t][i], (int32_t)e, l2g[t][cx_lq[t][i]]);
        x0 = ex_end[e];
      }
    };
    chunked(nt, (size_t)Ne, [&](int t, size_t lo, size_t hi) {
      int32_t *c = &ccnt[(size_t)t * Nn];
      chunk_entries(t, lo, hi, [&](int32_t n, int32_t, uint16_t) { c[n]++; });
    });
    m.dg_ptr.assign(Nn + 1, 0);
    chunked(host_threads(Nn), (size_t)Nn, [&](int, size_t lo, size_t hi) {
      for (size_t n = lo; n < hi; ++n) {
        int32_t s = 0;
        for (int t = 0; t < nt; ++t) s += ccnt[(size_t)t * Nn + n];
        m.dg_ptr[n + 1] = s;
      }
    });
    {
      int64_t run = 0;
      for (int64_t n = 0; n < Nn; ++n) {
        run += m.dg_ptr[n + 1];
        if (run > kMaxOffset) return kTooLarge;
        m.dg_ptr[n + 1] = (int32_t)run;
      }
    }
    chunked(host_threads(Nn), (size_t)Nn, [&](int, size_t lo, size_t hi) {
      for (size_t n = lo; n < hi; ++n) {
        int32_t s = m.dg_ptr[n];
        for (int t = 0; t < nt; ++t) {
          const int32_t v = ccnt[(size_t)t * Nn + n];
          ccnt[(size_t)t * Nn + n] = s;
          s += v;
        }
      }
    });
    m.dg_elem.resize(m.dg_ptr[Nn]);
    m.dg_q.resize(m.dg_ptr[Nn]);
    chunked(nt, (size_t)Ne, [&](int t, size_t lo, size_t hi) {
      int32_t *f = &ccnt[(size_t)t * Nn];
      chunk_entries(t, lo, hi, [&](int32_t n, int32_t e, uint16_t q) {
        m.dg_elem[f[n]] = e;
        m.dg_q[f[n]++] = q;
      });
    });
  }
  return "";
}

}  // namespace amr

// ---------------------------------------------------------------- host-only C ABI
struct tm_tables {
  amr::HostMesh m;
};

// The handler of the host-only entry points' function-try-blocks (inside a catch only): the status
// of the exception that would otherwise cross the C boundary, its message into err (err_len bytes).
static int table_exception(char *err, int err_len) noexcept {
  int code = TM_EINVAL;
  const char *what = "unexpected C++ exception";
  try {
    throw;
  } catch (const std::bad_alloc &) {
    code = TM_ENOMEM;
    what = "host memory allocation failed";
  } catch (const std::length_error &) {
    code = TM_ENOMEM;
    what = "host array size out of range";
  } catch (const std::exception &e) {
    what = e.what();
  } catch (...) {
  }
  if (err && err_len > 0) {
    std::strncpy(err, what, (size_t)err_len - 1);
    err[err_len - 1] = 0;
  }
  return code;
}

extern "C" {

int tm_tables_build(const tm_mesh_desc *d, tm_tables **out, tm_mesh_info *info, char *err, int err_len) try {
  if (!d || !out) return TM_EINVAL;
  *out = nullptr;
  std::unique_ptr<tm_tables> t(new tm_tables());
  std::string msg = amr::build_host_mesh(*d, t->m);
  if (!msg.empty()) {
    if (err && err_len > 0) {
      std::strncpy(err, msg.c_str(), (size_t)err_len - 1);
      err[err_len - 1] = 0;
    }
    return TM_EINVAL;
  }
  const amr::HostMesh &m = t->m;
  if (info) {
    info->Ne = m.Ne;
    info->Nn = m.Nn;
    info->n_hanging = (int64_t)m.hang_node.size();
    info->n_dirichlet = m.n_dirichlet;
    info->n_free = 3 * m.n_free_nodes;
    info->n_blocks = m.nblk;
    info->max_local = m.max_local;
    info->n_shared = (int64_t)m.sh_node.size();
    info->device_bytes = 0;
    info->max_block_bytes = m.max_rec_bytes;
    info->n_bricks = m.nbrick;
  }
  *out = t.release();
  return TM_OK;
} catch (...) {
  return table_exception(err, err_len);
}

int tm_tables_copy(const tm_tables *t, int64_t *perm, int32_t *node_xyz, int32_t *conn, int32_t *hang_node,
                   int32_t *hang_master, uint8_t *node_flags) try {
  if (!t) return TM_EINVAL;
  const amr::HostMesh &h = t->m;
  if (perm) std::memcpy(perm, h.perm.data(), h.perm.size() * sizeof(int64_t));
  if (node_xyz) std::memcpy(node_xyz, h.node_xyz.data(), h.node_xyz.size() * sizeof(int32_t));
  if (conn) std::memcpy(conn, h.conn.data(), h.conn.size() * sizeof(int32_t));
  if (hang_node) std::memcpy(hang_node, h.hang_node.data(), h.hang_node.size() * sizeof(int32_t));
  if (hang_master) std::memcpy(hang_master, h.hang_master.data(), h.hang_master.size() * sizeof(int32_t));
  if (node_flags) std::memcpy(node_flags, h.nflag.data(), h.nflag.size());
  return TM_OK;
} catch (...) {
  return table_exception(nullptr, 0);
}

int tm_tables_operator(const tm_tables *t, int32_t *rec_off, uint8_t *brec, double *modal, int32_t *sh_node,
                       int32_t *sh_ptr, int64_t *rec_bytes) try {
  if (!t) return TM_EINVAL;
  const amr::HostMesh &h = t->m;
  if (rec_bytes) *rec_bytes = (int64_t)h.brec.size();
  if (rec_off) std::memcpy(rec_off, h.rec_off.data(), h.rec_off.size() * sizeof(int32_t));
  if (brec) std::memcpy(brec, h.brec.data(), h.brec.size());
  if (modal) std::memcpy(modal, h.modal.data(), 72 * sizeof(double));
  if (sh_node) std::memcpy(sh_node, h.sh_node.data(), h.sh_node.size() * sizeof(int32_t));
  if (sh_ptr) std::memcpy(sh_ptr, h.sh_ptr.data(), h.sh_ptr.size() * sizeof(int32_t));
  return TM_OK;
} catch (...) {
  return table_exception(nullptr, 0);
}

int tm_tables_bricks(const tm_tables *t, int32_t *e0, int32_t *node, uint8_t *hax, int32_t *out, uint32_t *fold) try {
  if (!t) return TM_EINVAL;
  const amr::HostMesh &h = t->m;
  if (e0) std::memcpy(e0, h.brick_e0.data(), h.brick_e0.size() * sizeof(int32_t));
  if (node) std::memcpy(node, h.brick_node.data(), h.brick_node.size() * sizeof(int32_t));
  if (hax) std::memcpy(hax, h.brick_hax.data(), h.brick_hax.size());
  if (out) std::memcpy(out, h.brick_out.data(), h.brick_out.size() * sizeof(int32_t));
  if (fold) std::memcpy(fold, h.brick_fold.data(), h.brick_fold.size() * sizeof(uint32_t));
  return TM_OK;
} catch (...) {
  return table_exception(nullptr, 0);
}

int tm_tables_diag(const tm_tables *t, int32_t *ptr, int32_t *elem, uint16_t *q, double *tab, int64_t *n_entries,
                   int64_t *n_triples) try {
  if (!t) return TM_EINVAL;
  const amr::HostMesh &h = t->m;
  if (n_entries) *n_entries = (int64_t)h.dg_elem.size();
  if (n_triples) *n_triples = (int64_t)(h.dg_tab.size() / 3);
  if (ptr) std::memcpy(ptr, h.dg_ptr.data(), h.dg_ptr.size() * sizeof(int32_t));
  if (elem) std::memcpy(elem, h.dg_elem.data(), h.dg_elem.size() * sizeof(int32_t));
  if (q) std::memcpy(q, h.dg_q.data(), h.dg_q.size() * sizeof(uint16_t));
  if (tab) std::memcpy(tab, h.dg_tab.data(), h.dg_tab.size() * sizeof(double));
  return TM_OK;
} catch (...) {
  return table_exception(nullptr, 0);
}

int tm_tables_transfer(const tm_tables *t, const double *u_full, int64_t n_points, const int32_t *points,
                       double *out) try {
  if (!t || !u_full || (n_points > 0 && (!points || !out)) || n_points < 0) return TM_EINVAL;
  const amr::HostMesh &h = t->m;
  const int64_t fx = (int64_t)h.nx << h.L, fy = (int64_t)h.ny << h.L, fz = (int64_t)h.nz << h.L;
  for (int64_t i = 0; i < n_points; ++i) {
    const int64_t p[3] = {points[3 * i], points[3 * i + 1], points[3 * i + 2]};
    if (p[0] < 0 || p[1] < 0 || p[2] < 0 || p[0] > fx || p[1] > fy || p[2] > fz) return TM_EINVAL;
    // a cell whose closed box holds the point, and the leaf covering it
    const int64_t cx = std::min(p[0], fx - 1), cy = std::min(p[1], fy - 1), cz = std::min(p[2], fz - 1);
    const int64_t e = h.cellmap[(size_t)((cz * fy + cy) * fx + cx)];
    const int32_t *l = &h.leaf[4 * e];
    const double s = (double)(1 << (h.L - l[3]));
    const double tx = (p[0] - l[0]) / s, ty = (p[1] - l[1]) / s, tz = (p[2] - l[2]) / s;
    double v[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 8; ++k) {   // trilinear interpolation of the corner values
      const double w = ((k & 1) ? tx : 1.0 - tx) * (((k >> 1) & 1) ? ty : 1.0 - ty) * (((k >> 2) & 1) ? tz : 1.0 - tz);
      const double *uc = u_full + 3 * (size_t)h.conn[8 * e + k];
      v[0] += w * uc[0];
      v[1] += w * uc[1];
      v[2] += w * uc[2];
    }
    out[3 * i] = v[0];
    out[3 * i + 1] = v[1];
    out[3 * i + 2] = v[2];
  }
  return TM_OK;
} catch (...) {
  return table_exception(nullptr, 0);
}

void tm_tables_free(tm_tables *t) { delete t; }

}  // extern "C"

// ---------------------------------------------------------------- adaptation (paper Sec. 4)
namespace amr {

// New leaf set from final marks (+1 refine, 0 keep, -1 derefine; canonical order):
// refined leaves split into 8 children that inherit rho; a family of 8 siblings
// marked -1 (consecutive in Morton order) merges into its parent with the mean
// rho; then leaves are refined until every two touching leaves differ by at most
// one level (children inherit rho).
std::string adapt_leaves(const HostMesh &m, const int8_t *mark, const double *rho, std::vector<int32_t> &leaves,
                         std::vector<double> &rho_out) {
  const int L = m.L;
  const int64_t Ne = m.Ne;
  const int64_t fx = (int64_t)m.nx << L, fy = (int64_t)m.ny << L, fz = (int64_t)m.nz << L;
  // Every element's check and output depend on it and its family alone, so chunks of elements are
  // checked and counted in parallel, then write their outputs at the offsets of the earlier
  // chunks: the element order, and the first error in element order, of a sequential pass.
  auto check = [&](int64_t e) -> const char * {
    const int32_t *l = &m.leaf[4 * e];
    const int32_t s = 1 << (L - l[3]);
    if (mark[e] == 1) return l[3] >= L ? "refinement mark on a finest-level element" : nullptr;
    if (mark[e] != -1) return nullptr;
    if (l[3] == 0) return "derefinement mark on a level-0 element";
    const int32_t ps = 2 * s;
    const int k0 = (l[0] % ps ? 1 : 0) + (l[1] % ps ? 2 : 0) + (l[2] % ps ? 4 : 0);
    if (k0) {   // merged with the family's first sibling, which must carry the same mark
      const int32_t *f = e >= k0 ? &m.leaf[4 * (e - k0)] : nullptr;
      if (!f || f[3] != l[3] || f[0] != l[0] - s * (k0 & 1) || f[1] != l[1] - s * ((k0 >> 1) & 1) ||
          f[2] != l[2] - s * ((k0 >> 2) & 1) || mark[e - k0] != -1)
        return "family marked for derefinement is not 8 sibling leaves";
      return nullptr;
    }
    if (e + 8 > Ne) return "incomplete family marked for derefinement";
    for (int k = 0; k < 8; ++k) {
      const int32_t *q = &m.leaf[4 * (e + k)];
      if (mark[e + k] != -1 || q[3] != l[3] || q[0] != l[0] + s * (k & 1) || q[1] != l[1] + s * ((k >> 1) & 1) ||
          q[2] != l[2] + s * ((k >> 2) & 1))
        return "family marked for derefinement is not 8 sibling leaves";
    }
    return nullptr;
  };
  auto count = [&](int64_t e) -> int64_t {
    if (mark[e] == 1) return 8;
    if (mark[e] == -1) {
      const int32_t *l = &m.leaf[4 * e];
      const int32_t ps = 2 << (L - l[3]);
      return l[0] % ps || l[1] % ps || l[2] % ps ? 0 : 1;
    }
    return 1;
  };
  const int nt = host_threads(Ne);
  std::vector<int64_t> off(nt + 1, 0);
  std::vector<const char *> err(nt, nullptr);
  chunked(nt, (size_t)Ne, [&](int t, size_t lo, size_t hi) {
    int64_t c = 0;
    for (size_t e = lo; e < hi; ++e) {
      if ((err[t] = check((int64_t)e))) return;
      c += count((int64_t)e);
    }
    off[t + 1] = c;
  });
  for (int t = 0; t < nt; ++t)
    if (err[t]) return err[t];
  for (int t = 0; t < nt; ++t) off[t + 1] += off[t];
  leaves.assign(4 * (size_t)off[nt], 0);
  rho_out.assign((size_t)off[nt], 0.0);
  chunked(nt, (size_t)Ne, [&](int t, size_t lo, size_t hi) {
    int64_t o = off[t];
    for (size_t e = lo; e < hi; ++e) {
      const int32_t *l = &m.leaf[4 * e];
      const int32_t s = 1 << (L - l[3]);
      if (mark[e] == 1) {
        const int32_t h = s / 2;
        for (int k = 0; k < 8; ++k, ++o) {
          int32_t *q = &leaves[4 * o];
          q[0] = l[0] + h * (k & 1); q[1] = l[1] + h * ((k >> 1) & 1); q[2] = l[2] + h * ((k >> 2) & 1); q[3] = l[3] + 1;
          rho_out[o] = rho[e];
        }
      } else if (mark[e] == -1) {
        if (!count((int64_t)e)) continue;
        double sum = 0.0;
        for (int k = 0; k < 8; ++k) sum += rho[e + k];
        int32_t *q = &leaves[4 * o];
        q[0] = l[0]; q[1] = l[1]; q[2] = l[2]; q[3] = l[3] - 1;
        rho_out[o++] = sum / 8.0;
      } else {
        std::memcpy(&leaves[4 * o], l, 16);
        rho_out[o++] = rho[e];
      }
    }
  });
  // 2:1 balance by refinement: paint every leaf's level into the finest cells (leaves are
  // disjoint, so the threads write disjoint cells), then split every leaf that touches -- across
  // a face, an edge or a corner -- a leaf more than one level finer
  std::vector<uint8_t> lv((size_t)(fx * fy * fz));
  for (int pass = 0; pass < 64; ++pass) {
    const int64_t n = (int64_t)rho_out.size();
    const int nb = host_threads(n);
    chunked(nb, (size_t)n, [&](int, size_t lo, size_t hi) {
      for (size_t i = lo; i < hi; ++i) {
        const int32_t *l = &leaves[4 * i];
        const int32_t s = 1 << (L - l[3]);
        for (int z = 0; z < s; ++z)
          for (int y = 0; y < s; ++y)
            std::memset(&lv[((size_t)(l[2] + z) * fy + (l[1] + y)) * fx + l[0]], l[3], s);
      }
    });
    std::vector<uint8_t> need(n, 0);
    std::vector<int64_t> noff(nb + 1, 0);
    chunked(nb, (size_t)n, [&](int t, size_t lo, size_t hi) {
      int64_t c = 0;
      for (size_t i = lo; i < hi; ++i) {
        const int32_t *l = &leaves[4 * i];
        const int64_t s = (int64_t)1 << (L - l[3]);
        const int64_t x0 = std::max<int64_t>(l[0] - 1, 0), x1 = std::min<int64_t>(l[0] + s + 1, fx);
        int mx = 0;
        for (int64_t z = std::max<int64_t>(l[2] - 1, 0); z < std::min<int64_t>(l[2] + s + 1, fz); ++z)
          for (int64_t y = std::max<int64_t>(l[1] - 1, 0); y < std::min<int64_t>(l[1] + s + 1, fy); ++y) {
            const uint8_t *row = &lv[((size_t)z * fy + y) * fx];
            if (z >= l[2] && z < l[2] + s && y >= l[1] && y < l[1] + s) {   // the leaf's own rows: both ends
              if (l[0] - 1 >= 0) mx = std::max<int>(mx, row[l[0] - 1]);
              if (l[0] + s < fx) mx = std::max<int>(mx, row[l[0] + s]);
            } else {
              for (int64_t x = x0; x < x1; ++x) mx = std::max<int>(mx, row[x]);
            }
          }
        need[i] = mx > l[3] + 1;
        c += need[i] ? 8 : 1;
      }
      noff[t + 1] = c;
    });
    for (int t = 0; t < nb; ++t) noff[t + 1] += noff[t];
    if (noff[nb] == n) return "";
    std::vector<int32_t> nl(4 * (size_t)noff[nb]);
    std::vector<double> nr((size_t)noff[nb]);
    chunked(nb, (size_t)n, [&](int t, size_t lo, size_t hi) {
      int64_t o = noff[t];
      for (size_t i = lo; i < hi; ++i) {
        const int32_t *l = &leaves[4 * i];
        if (!need[i]) {
          std::memcpy(&nl[4 * o], l, 16);
          nr[o++] = rho_out[i];
          continue;
        }
        const int32_t h = (1 << (L - l[3])) / 2;
        for (int k = 0; k < 8; ++k, ++o) {
          int32_t *q = &nl[4 * o];
          q[0] = l[0] + h * (k & 1); q[1] = l[1] + h * ((k >> 1) & 1); q[2] = l[2] + h * ((k >> 2) & 1); q[3] = l[3] + 1;
          nr[o] = rho_out[i];
        }
      }
    });
    leaves.swap(nl);
    rho_out.swap(nr);
  }
  return "2:1 balancing did not settle";
}

}  // namespace amr

extern "C" {

int tm_tables_adapt(const tm_tables *t, const int8_t *mark, const double *rho, int64_t capacity,
                    int32_t *leaves_out, double *rho_out, int64_t *n_out) try {
  if (!t || !mark || !rho || !n_out) return TM_EINVAL;
  std::vector<int32_t> lv;
  std::vector<double> r;
  if (!amr::adapt_leaves(t->m, mark, rho, lv, r).empty()) return TM_EINVAL;
  *n_out = (int64_t)r.size();
  if ((int64_t)r.size() > capacity || !leaves_out || !rho_out) return TM_EINVAL;
  std::memcpy(leaves_out, lv.data(), lv.size() * sizeof(int32_t));
  std::memcpy(rho_out, r.data(), r.size() * sizeof(double));
  return TM_OK;
} catch (...) {
  return table_exception(nullptr, 0);
}

}  // extern "C"
