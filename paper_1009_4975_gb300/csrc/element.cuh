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

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// FP32: components 0 and 1 of every corner travel as one packed pair through the butterflies and
// the coefficient scaling (add.rn.f32x2 / fma.rn.f32x2: each half rounds as its scalar
// counterpart), component 2 as a scalar; the 3x3 blocks are scalar FMA chains.
template <int MODE>
__device__ __forceinline__ float element_op_f32x2(const float X[24], float Y[24], float coef,
                                                  const ModalBlocks<float> &M) {
  constexpr bool WANT_ENERGY = MODE != kOpApply;
  constexpr bool WANT_Y = MODE != kOpEnergy;
  const float2 neg1 = make_float2(-1.f, -1.f);
  float2 p[8];
  float z[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    p[k] = make_float2(X[3 * k], X[3 * k + 1]);
    z[k] = X[3 * k + 2];
  }
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (!(k & bit)) {
        const float2 a = p[k], b = p[k | bit];
        p[k] = __fadd2_rn(a, b);
        p[k | bit] = __ffma2_rn(a, neg1, b);     // b - a
        const float c = z[k], d = z[k | bit];
        z[k] = c + d;
        z[k | bit] = d - c;
      }
  float2 qp[8];
  float qz[8];
  float energy = 0.f;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const float a0 = p[s ^ 1].x, a1 = p[s ^ 2].y, a2 = z[s ^ 4];
    float r0, r1, r2;
    if (s == 1) {        // component 0 of this block is a translation
      r0 = 0.f;
      r1 = fmaf(M.b[s][1][2], a2, M.b[s][1][1] * a1);
      r2 = fmaf(M.b[s][2][2], a2, M.b[s][2][1] * a1);
    } else if (s == 2) {
      r0 = fmaf(M.b[s][0][2], a2, M.b[s][0][0] * a0);
      r1 = 0.f;
      r2 = fmaf(M.b[s][2][2], a2, M.b[s][2][0] * a0);
    } else if (s == 4) {
      r0 = fmaf(M.b[s][0][1], a1, M.b[s][0][0] * a0);
      r1 = fmaf(M.b[s][1][1], a1, M.b[s][1][0] * a0);
      r2 = 0.f;
    } else {
      r0 = fmaf(M.b[s][0][2], a2, fmaf(M.b[s][0][1], a1, M.b[s][0][0] * a0));
      r1 = fmaf(M.b[s][1][2], a2, fmaf(M.b[s][1][1], a1, M.b[s][1][0] * a0));
      r2 = fmaf(M.b[s][2][2], a2, fmaf(M.b[s][2][1], a1, M.b[s][2][0] * a0));
    }
    if (WANT_ENERGY) energy = fmaf(a2, r2, fmaf(a1, r1, fmaf(a0, r0, energy)));
    if (WANT_Y) {
      qp[s ^ 1].x = r0;
      qp[s ^ 2].y = r1;
      qz[s ^ 4] = r2;
    }
  }
  if (!WANT_Y) return energy;
  const float2 cc = make_float2(coef, coef);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    qp[k] = __fmul2_rn(qp[k], cc);
    qz[k] *= coef;
  }
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (!(k & bit)) {
        const float2 sv = qp[k], dv = qp[k | bit];
        qp[k] = __ffma2_rn(dv, neg1, sv);       // s - d
        qp[k | bit] = __fadd2_rn(sv, dv);
        const float c = qz[k], d = qz[k | bit];
        qz[k] = c - d;
        qz[k | bit] = c + d;
      }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    Y[3 * k] = qp[k].x;
    Y[3 * k + 1] = qp[k].y;
    Y[3 * k + 2] = qz[k];
  }
  return WANT_ENERGY ? coef * energy : 0.f;
}
#endif

template <typename T, int MODE>
__device__ __forceinline__ T element_op(const T X[24], T Y[24], T coef, const ModalBlocks<T> &M) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  if constexpr (sizeof(T) == 4) return element_op_f32x2<MODE>(X, Y, coef, M);
#endif
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
