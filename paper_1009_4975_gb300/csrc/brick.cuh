// The brick pass of the operator (paper Eq. 6-9 on a brick): y = C^T K(rho) C x restricted to
// the 64 elements of an aligned 4x4x4 cube of equal-level elements (mesh_host.cpp, section 6a).
// The brick's 5x5x5 node lattice replaces the per-block record: node (a, b, c) is staged at
// a + 8 b + 68 c of a per-component array (pitches for which the 32 elements of a warp, a
// 4 x 4 x 2 sub-cube, read 32 distinct banks for every corner).  Thread t of the brick's 64 takes
// element (i, j, k) = (t % 4, t / 4 % 4, t / 16), which is element e0 + morton(i, j, k).  Steps:
//   0. the brick's packed table (node ids and e0, output targets, fold masks and axes; 1.5 KB)
//      into shared memory with 16-byte copies;
//   1. regular lattice nodes: their values (zero at Dirichlet nodes), and the 64 coefficients;
//   2. hanging lattice nodes (bricks next to coarser elements only): the (bi)linear
//      interpolation of their masters (C), the lattice nodes one step away along the axes of the
//      coarse edge or face;
//   3. one thread per element: Y = c_e K0 X_e (element.cuh), kept in registers;
//   4. node sums without a result buffer: along x each thread adds the x-upper corners of the
//      element before it (shuffle by one lane), then along y (by four lanes), then along z (by
//      sixteen lanes; the plane between the brick's two warps through shared memory), so that
//      the lower corner of every element, and the upper corners of the elements on the brick's
//      upper faces, hold complete node sums, which are stored over the node values;
//   5. regular nodes add w times the sums of the hanging nodes they are masters of (C^T; the
//      neighbours named by the node's fold mask in bit order, w = 1/2 along an edge, 1/4 on a
//      face), and store to y (nodes only this brick touches) or to their partial slots; hanging
//      nodes store nothing (their DOFs of y are zeroed by the shared-node pass).
// The arithmetic is fixed by the brick alone, so the single- and multi-vector passes agree bit
// for bit.  Each brick synchronises its own 64 threads (named barriers), so the four bricks of a
// CTA proceed independently.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "element.cuh"

namespace amr {

constexpr int kBrickElems = 64;
constexpr int kBrickNodes = 125;
constexpr int kBricksPerCta = 4;
constexpr int kLatY = 8, kLatZ = 68;
constexpr int kLatPitch = 312;           // >= 4 + 4 kLatY + 4 kLatZ + 1, multiple of 4

// Device table of the bricks: per brick 3 x 128 int32 -- [0, 125) lattice node ids (bit 31
// Dirichlet) and e0 at 125; [128, 253) output targets (-1 owned, >= 0 partial slot, -2 hanging);
// [256, 381) fold mask (bits 0-17) | interpolation axes of a hanging node << 24.
constexpr int kBrickTab = 384;
struct BrickTables {
  const int32_t *tab;
  int nbrick;
};

// per brick: 3 x kLatPitch node values, 16 x 12 values of the plane between its warps, the 64
// coefficients, the table
template <typename T>
__host__ __device__ __forceinline__ size_t brick_bytes() {
  return (3 * kLatPitch + 16 * 12 + kBrickElems) * sizeof(T) + kBrickTab * sizeof(int32_t);
}
template <typename T>
__host__ __device__ __forceinline__ size_t brick_smem_bytes() {
  return (size_t)kBricksPerCta * brick_bytes<T>();
}

// Barriers of one brick's 64 threads (named barrier 1 + group; barrier 0 is __syncthreads), so
// that the bricks of a CTA do not wait for one another.
__device__ __forceinline__ void brick_sync(int g) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "r"(kBrickElems) : "memory");
}
__device__ __forceinline__ bool brick_sync_or(int g, bool v) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(out)
      : "r"((uint32_t)v), "r"(1 + g), "r"(kBrickElems)
      : "memory");
  return out != 0;
}

__device__ __forceinline__ void brick_cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}

__device__ __forceinline__ int brick_lat(int a, int b, int c) { return a + kLatY * b + kLatZ * c; }
__device__ __forceinline__ int brick_morton(int i, int j, int k) {
  return (i & 1) | ((j & 1) << 1) | ((k & 1) << 2) | ((i & 2) << 2) | ((j & 2) << 3) | ((k & 2) << 4);
}

__device__ __forceinline__ uint32_t brick_smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
template <int BYTES>
__device__ __forceinline__ void brick_cp_async(void *dst, const void *src, bool fill_zero) {
  const int srcsz = fill_zero ? 0 : BYTES;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(brick_smem_u32(dst)), "l"(src), "n"(BYTES),
               "r"(srcsz)
               : "memory");
}

// One brick per 64-thread group of a 256-thread CTA; `brick` may be past the last brick (the
// group then only takes part in the barriers).  Returns the thread's element energy
// c_e X_e^T K0 X_e when ENERGY, else 0.
template <typename T, bool ENERGY>
__device__ double brick_pass(const BrickTables &B, int brick, const T *ce, const T *x, T *y, T *part,
                             const ModalBlocks<T> &K, unsigned char *smem) {
  const int g = threadIdx.x / kBrickElems, lt = threadIdx.x % kBrickElems;
  unsigned char *base = smem + (size_t)g * brick_bytes<T>();
  T *R = reinterpret_cast<T *>(base);                           // 3 x kLatPitch, component-major
  T *Zp = R + 3 * kLatPitch;                                    // 16 x 12: plane between the warps
  T *cs = Zp + 16 * 12;                                         // 64 coefficients, element order
  int32_t *tab = reinterpret_cast<int32_t *>(cs + kBrickElems); // kBrickTab
  const bool valid = brick < B.nbrick;
  // the thread's lattice nodes lt and lt + 64 (the latter when < 125) and their offsets
  int Lnd[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int nd = lt + r * kBrickElems, c = nd / 25, rr = nd - 25 * c, b = rr / 5;
    Lnd[r] = brick_lat(rr - 5 * b, b, c);
  }
  // 0. the table
  if (valid) {
    const int4 *src = reinterpret_cast<const int4 *>(B.tab + (size_t)kBrickTab * brick);
    for (int w = lt; w < kBrickTab / 4; w += kBrickElems) brick_cp16(tab + 4 * w, src + w);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  brick_sync(g);
  // 1. node values of the regular lattice nodes, and the coefficients
  bool hang = false;
  if (valid) {
    // e0 need not be a multiple of 4: element-sized copies
    brick_cp_async<sizeof(T)>(cs + lt, ce + tab[125] + lt, false);
#pragma unroll
    for (int rn = 0; rn < 2; ++rn) {
      const int nd = lt + rn * kBrickElems;
      if (nd >= kBrickNodes) break;
      const int h = (uint32_t)tab[256 + nd] >> 24;
      hang |= h != 0;
      if (h) continue;
      const int L0 = Lnd[rn];
      const uint32_t gw = (uint32_t)tab[nd];
      const T *src = x + 3 * (size_t)(gw & 0x7FFFFFFFu);
      const bool zero = (gw >> 31) != 0;
#pragma unroll
      for (int q = 0; q < 3; ++q) brick_cp_async<sizeof(T)>(R + q * kLatPitch + L0, src + q, zero);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  hang = brick_sync_or(g, hang);         // the brick is next to coarser elements
  // 2. hanging lattice nodes from their masters
  if (hang) {
    if (valid)
#pragma unroll
      for (int rn = 0; rn < 2; ++rn) {
        const int nd = lt + rn * kBrickElems;
        if (nd >= kBrickNodes) break;
        const int m = (uint32_t)tab[256 + nd] >> 24;
        if (!m) continue;
        const int L0 = Lnd[rn];
        const int da = (m & 1) ? 1 : ((m & 2) ? kLatY : kLatZ);  // first axis of the mask
        const int db = (m & 4) ? kLatZ : kLatY;                  // last axis of the mask
        const bool edge = m == 1 || m == 2 || m == 4;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const T *rr = R + q * kLatPitch + L0;
          R[q * kLatPitch + L0] = edge ? T(0.5) * (rr[-da] + rr[da])   // an edge: da is its axis
                                       : T(0.25) * ((rr[-da - db] + rr[da - db]) + (rr[-da + db] + rr[da + db]));
        }
      }
    brick_sync(g);
  }
  // 3. element products (registers)
  const int i = lt & 3, j = (lt >> 2) & 3, k = lt >> 4;
  T Y[24];
  double energy = 0.0;
  if (valid) {
    const int L0 = brick_lat(i, j, k);
    T X[24];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int o = L0 + (q & 1) + kLatY * ((q >> 1) & 1) + kLatZ * (q >> 2);
#pragma unroll
      for (int c = 0; c < 3; ++c) X[3 * q + c] = R[c * kLatPitch + o];
    }
    const T coef = cs[brick_morton(i, j, k)];
    if (ENERGY) energy = (double)element_op<T, kOpBoth>(X, Y, coef, K);
    else element_op<T, kOpApply>(X, Y, coef, K);
  } else {
#pragma unroll
    for (int q = 0; q < 24; ++q) Y[q] = T(0);
  }
  // 4. node sums: corner q = dx + 2 dy + 4 dz
#pragma unroll
  for (int q = 0; q < 8; q += 2)           // x: the x-lower corners take the previous element's x-upper
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T v = __shfl_up_sync(0xffffffffu, Y[3 * (q + 1) + c], 1);
      if (i > 0) Y[3 * q + c] += v;
    }
#pragma unroll
  for (int q = 0; q < 8; ++q) {            // y: corners with dy = 0 (q & 2 clear)
    if (q & 2) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T v = __shfl_up_sync(0xffffffffu, Y[3 * (q + 2) + c], 4);
      if (j > 0) Y[3 * q + c] += v;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)              // z within the warp: corners with dz = 0
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T v = __shfl_up_sync(0xffffffffu, Y[3 * (q + 4) + c], 16);
      if (k & 1) Y[3 * q + c] += v;
    }
  if (k == 1)                              // the plane k = 2: the first warp's part
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) Zp[(lt - 16) * 12 + 3 * q + c] = Y[3 * (q + 4) + c];
  brick_sync(g);                           // also: every element has read its corners
  if (k == 2)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[3 * q + c] += Zp[(lt - 32) * 12 + 3 * q + c];
  // the corners holding complete sums: the lower corner, and upper corners on the brick's upper
  // faces; stored over the node values
  if (valid)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int dx = q & 1, dy = (q >> 1) & 1, dz = q >> 2;
      if ((dx && i != 3) || (dy && j != 3) || (dz && k != 3)) continue;
      const int L0 = brick_lat(i + dx, j + dy, k + dz);
#pragma unroll
      for (int c = 0; c < 3; ++c) R[c * kLatPitch + L0] = Y[3 * q + c];
    }
  brick_sync(g);
  // 5. folds of the hanging sums into their masters, then the stores
  if (valid)
#pragma unroll
    for (int rn = 0; rn < 2; ++rn) {
      const int nd = lt + rn * kBrickElems;
      if (nd >= kBrickNodes) break;
      const uint32_t fh = (uint32_t)tab[256 + nd];
      if (fh >> 24) continue;
      const int L0 = Lnd[rn];
      T s0 = R[L0], s1 = R[kLatPitch + L0], s2 = R[2 * kLatPitch + L0];
      if (hang) {
        uint32_t fm = fh & 0xFFFFFFu;
        while (fm) {
          const int bit = __ffs(fm) - 1;
          fm &= fm - 1;
          int o;
          T w;
          if (bit < 6) {
            const int ax = bit >> 1, sg = (bit & 1) ? 1 : -1;
            o = sg * (ax == 0 ? 1 : (ax == 1 ? kLatY : kLatZ));
            w = T(0.5);
          } else {
            const int bb = bit - 6, pl = bb >> 2;
            const int s0g = (bb & 1) ? 1 : -1, s1g = (bb & 2) ? 1 : -1;
            const int st0 = pl == 2 ? kLatY : 1, st1 = pl == 0 ? kLatY : kLatZ;
            o = s0g * st0 + s1g * st1;
            w = T(0.25);
          }
          s0 += w * R[L0 + o]; s1 += w * R[kLatPitch + L0 + o]; s2 += w * R[2 * kLatPitch + L0 + o];
        }
      }
      const uint32_t gw = (uint32_t)tab[nd];
      if (gw >> 31) s0 = s1 = s2 = T(0);
      const int ot = tab[128 + nd];
      T *dst = ot >= 0 ? part + 3 * (size_t)ot : y + 3 * (size_t)(gw & 0x7FFFFFFFu);
      dst[0] = s0; dst[1] = s1; dst[2] = s2;
    }
  return energy;
}

}  // namespace amr
