// The B8 element operator y_e = c * K0 x_e on the unit cube in a symmetry-adapted
// basis.
//
// Along each axis, the pair of nodal values (u at t = 0, u at t = 1) is replaced by
// its sum and difference; over the three axes this is a 3-stage butterfly
// w = T x per displacement component (T has entries +-1, T T^T = 8 I).  The unit
// cube with isotropic material is invariant under the reflection of each axis,
// and in the butterfly basis each modal DOF (component c, mode bits b) is even or
// odd under the three reflections (signature s, with bit a set when odd: b_a XOR
// [a == c]).  K0 commutes with the reflections, so K0m = T K0 T^T / 64 only couples
// DOFs of equal signature: eight 3x3 blocks, DOF c of block s being mode s ^ (1 << c).
// The three blocks s = 1, 2, 4 contain a rigid translation (mode 0 of component
// log2 s), whose row and column vanish; they act as 2x2 blocks.
//
//   y = c * T^T (K0m (T x))  -- ~72 add/sub forward, 57 FMA in the blocks,
//                              ~72 add/sub back: ~220 flops instead of 1152 dense.
//
// Differences along each axis cancel rigid translations before any rounding.
// K0m is computed on the host from the element matrix (mesh_host.cpp) and passed
// in the kernel parameters.
#pragma once

template <typename T>
struct ModalBlocks {
  T b[8][3][3];   // [signature s][row c][column c']
};

// In-place butterfly of 8 values along bit `bit`: (v0, v1) -> (v0 + v1, v1 - v0).
template <typename T>
__device__ __forceinline__ void fwd_stage(T v[8], int bit) {
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!(k & bit)) {
      const T a = v[k], b = v[k | bit];
      v[k] = a + b;
      v[k | bit] = b - a;
    }
}
// Transposed butterfly: (s, d) -> (s - d, s + d).
template <typename T>
__device__ __forceinline__ void bwd_stage(T v[8], int bit) {
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (!(k & bit)) {
      const T s = v[k], d = v[k | bit];
      v[k] = s - d;
      v[k | bit] = s + d;
    }
}

// X, Y: 24 values, DOF 3*k + c of corner k = i + 2j + 4m.
// MODE 0: writes Y = coef K0 X.  MODE 1: returns X^T K0 X (Y untouched).
// MODE 2: both, returning coef X^T K0 X (a sum of per-block quadratic forms of
// positive semidefinite blocks, free of the cancellation of X . Y).
constexpr int kOpApply = 0, kOpEnergy = 1, kOpBoth = 2;
template <typename T, int MODE>
__device__ __forceinline__ T element_op(const T X[24], T Y[24], T coef, const ModalBlocks<T> &M) {
  constexpr bool WANT_ENERGY = MODE != kOpApply;
  constexpr bool WANT_Y = MODE != kOpEnergy;
  T w[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int k = 0; k < 8; ++k) w[c][k] = X[3 * k + c];
    fwd_stage<T>(w[c], 1);
    fwd_stage<T>(w[c], 2);
    fwd_stage<T>(w[c], 4);
  }
  T z[3][8];
  T energy = T(0);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const T a0 = w[0][s ^ 1], a1 = w[1][s ^ 2], a2 = w[2][s ^ 4];
    T r0, r1, r2;
    if (s == 1) {        // component 0 of this block is a translation
      r0 = T(0);
      r1 = M.b[s][1][1] * a1 + M.b[s][1][2] * a2;
      r2 = M.b[s][2][1] * a1 + M.b[s][2][2] * a2;
    } else if (s == 2) {
      r0 = M.b[s][0][0] * a0 + M.b[s][0][2] * a2;
      r1 = T(0);
      r2 = M.b[s][2][0] * a0 + M.b[s][2][2] * a2;
    } else if (s == 4) {
      r0 = M.b[s][0][0] * a0 + M.b[s][0][1] * a1;
      r1 = M.b[s][1][0] * a0 + M.b[s][1][1] * a1;
      r2 = T(0);
    } else {
      r0 = M.b[s][0][0] * a0 + M.b[s][0][1] * a1 + M.b[s][0][2] * a2;
      r1 = M.b[s][1][0] * a0 + M.b[s][1][1] * a1 + M.b[s][1][2] * a2;
      r2 = M.b[s][2][0] * a0 + M.b[s][2][1] * a1 + M.b[s][2][2] * a2;
    }
    if (WANT_ENERGY) energy += a0 * r0 + a1 * r1 + a2 * r2;
    if (WANT_Y) {
      z[0][s ^ 1] = r0;
      z[1][s ^ 2] = r1;
      z[2][s ^ 4] = r2;
    }
  }
  if (!WANT_Y) return energy;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int k = 0; k < 8; ++k) z[c][k] *= coef;
    bwd_stage<T>(z[c], 1);
    bwd_stage<T>(z[c], 2);
    bwd_stage<T>(z[c], 4);
#pragma unroll
    for (int k = 0; k < 8; ++k) Y[3 * k + c] = z[c][k];
  }
  return WANT_ENERGY ? coef * energy : T(0);
}
