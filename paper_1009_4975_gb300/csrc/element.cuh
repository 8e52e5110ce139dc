// The B8 element operator y_e = c * K0 x_e on the unit cube, evaluated by sum
// factorisation over the 2x2x2 Gauss points instead of a dense 24x24 product.
//
// K0 = sum_q w_q B_q^T D B_q (w_q = 1/8).  For trilinear shape functions
// N_ijk = f_i(x) f_j(y) f_k(z) (f_0 = 1 - t, f_1 = t) the displacement gradient at
// a Gauss point is a tensor product of 2x2 interpolations of edge differences:
//   du_c/dx (a,b,d) = sum_{j,k} M[b][j] M[d][k] (u_c(1,j,k) - u_c(0,j,k))
// with M[a][i] = f_i(g_a), g_{0,1} = (1 -/+ 1/sqrt3)/2, and symmetrically for
// y and z.  Stresses follow from isotropic Hooke's law (Lame constants of
// E = 1); the transpose B^T sigma folds back through the same M (symmetric).
// Cost: ~580 flops per element against 1152 for the dense product, and the
// edge differences remove rigid translations before any rounding.
#pragma once

template <typename T>
struct GaussM {
  static constexpr double g0 = 0.21132486540518711775;  // (1 - 1/sqrt(3)) / 2
  static constexpr double g1 = 0.78867513459481288225;  // (1 + 1/sqrt(3)) / 2
};

// out[P][Q] = sum_{p,q} M[P][p] M[Q][q] in[p][q]
template <typename T>
__device__ __forceinline__ void interp2(const T in[2][2], T out[2][2]) {
  const T g0 = T(GaussM<T>::g0), g1 = T(GaussM<T>::g1);
  T t00 = g1 * in[0][0] + g0 * in[0][1];
  T t01 = g0 * in[0][0] + g1 * in[0][1];
  T t10 = g1 * in[1][0] + g0 * in[1][1];
  T t11 = g0 * in[1][0] + g1 * in[1][1];
  out[0][0] = g1 * t00 + g0 * t10;
  out[1][0] = g0 * t00 + g1 * t10;
  out[0][1] = g1 * t01 + g0 * t11;
  out[1][1] = g0 * t01 + g1 * t11;
}

// X, Y: 24 values, DOF 3*k + c of corner k = i + 2j + 4m.
// Returns u^T K0 u when WANT_ENERGY (Y then untouched); else writes Y = c K0 X.
template <typename T, bool WANT_ENERGY>
__device__ __forceinline__ T element_op(const T X[24], T Y[24], T coef, T lam, T mu) {
  T Gx[3][2][2], Gy[3][2][2], Gz[3][2][2];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T dx[2][2], dy[2][2], dz[2][2];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        dx[p][q] = X[3 * (1 + 2 * p + 4 * q) + c] - X[3 * (0 + 2 * p + 4 * q) + c];  // [j][k]
        dy[p][q] = X[3 * (p + 2 * 1 + 4 * q) + c] - X[3 * (p + 2 * 0 + 4 * q) + c];  // [i][k]
        dz[p][q] = X[3 * (p + 2 * q + 4 * 1) + c] - X[3 * (p + 2 * q + 4 * 0) + c];  // [i][j]
      }
    interp2<T>(dx, Gx[c]);  // [b][d]
    interp2<T>(dy, Gy[c]);  // [a][d]
    interp2<T>(dz, Gz[c]);  // [a][b]
  }
  T Sx[3][2][2], Sy[3][2][2], Sz[3][2][2];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) Sx[c][p][q] = Sy[c][p][q] = Sz[c][p][q] = T(0);
  T energy = T(0);
  const T two_mu = mu + mu;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const T exx = Gx[0][b][d], eyy = Gy[1][a][d], ezz = Gz[2][a][b];
        const T gxy = Gy[0][a][d] + Gx[1][b][d];
        const T gyz = Gz[1][a][b] + Gy[2][a][d];
        const T gzx = Gx[2][b][d] + Gz[0][a][b];
        const T ltr = lam * (exx + eyy + ezz);
        const T sxx = ltr + two_mu * exx, syy = ltr + two_mu * eyy, szz = ltr + two_mu * ezz;
        const T sxy = mu * gxy, syz = mu * gyz, szx = mu * gzx;
        if (WANT_ENERGY) {
          energy += sxx * exx + syy * eyy + szz * ezz + sxy * gxy + syz * gyz + szx * gzx;
        } else {
          Sx[0][b][d] += sxx; Sy[0][a][d] += sxy; Sz[0][a][b] += szx;
          Sx[1][b][d] += sxy; Sy[1][a][d] += syy; Sz[1][a][b] += syz;
          Sx[2][b][d] += szx; Sy[2][a][d] += syz; Sz[2][a][b] += szz;
        }
      }
  if (WANT_ENERGY) return energy * T(0.125);
  const T w = coef * T(0.125);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T tx[2][2], ty[2][2], tz[2][2];
    interp2<T>(Sx[c], tx);  // [j][k]
    interp2<T>(Sy[c], ty);  // [i][k]
    interp2<T>(Sz[c], tz);  // [i][j]
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = k & 1, j = (k >> 1) & 1, m = (k >> 2) & 1;
      const T v = (i ? tx[j][m] : -tx[j][m]) + (j ? ty[i][m] : -ty[i][m]) + (m ? tz[i][j] : -tz[i][j]);
      Y[3 * k + c] = w * v;
    }
  }
  return T(0);
}
