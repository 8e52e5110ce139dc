/* Oracle CPU baseline: FP64 Jacobi-preconditioned CG on an assembled CSR matrix, with OpenMP
 * threads for the sparse matrix-vector product, the vector updates and the dot products.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): it is the timed CPU baseline of the
 * benchmark and is never part of the library's path.
 *
 * The algorithm is the textbook preconditioned CG with the diagonal of A as preconditioner
 * (the symmetric rescaling D^-1/2 A D^-1/2 of the paper's Sec. 5 applied implicitly): r = f - A u,
 * z = D^-1 r, p = z; repeat q = A p, alpha = r.z / p.q, u += alpha p, r -= alpha q,
 * z = D^-1 r, beta = r.z' / r.z, p = z + beta p, until ||r|| <= rtol ||f||.  Dot products are
 * OpenMP reductions (their summation order depends on the thread count).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static void spmv(int64_t n, const int64_t *ptr, const int32_t *col, const double *val, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = s;
  }
}

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Returns the iterations performed (max_iter when not converged); *rel receives the final
 * recurrence ||r|| / ||f||.  Work vectors r, z, p, q (n each) are caller-provided; u holds the
 * initial guess on entry and the solution on exit. */
int64_t oracle_jacobi_pcg(int64_t n, const int64_t *ptr, const int32_t *col, const double *val, const double *f,
                          double *u, double rtol, int64_t max_iter, double *r, double *z, double *p, double *q,
                          double *rel) {
  double *dinv = q;   /* the diagonal's inverse lives in q until the first product */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k)
      if (col[k] == i) d = val[k];
    dinv[i] = 1.0 / d;
  }
  /* z holds D^-1 during the iteration; r = f - A u */
  memcpy(z, dinv, (size_t)n * sizeof(double));
  spmv(n, ptr, col, val, u, p);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) r[i] = f[i] - p[i];
  const double fn = sqrt(dot(n, f, f));
  double rz = 0.0;
#pragma omp parallel for reduction(+ : rz) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    p[i] = z[i] * r[i];
    rz += r[i] * p[i];
  }
  double rn = sqrt(dot(n, r, r));
  int64_t it = 0;
  while (rn > rtol * fn && it < max_iter) {
    spmv(n, ptr, col, val, p, q);
    const double alpha = rz / dot(n, p, q);
    double rz_new = 0.0, rr = 0.0;
#pragma omp parallel for reduction(+ : rz_new, rr) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      u[i] += alpha * p[i];
      r[i] -= alpha * q[i];
      rz_new += r[i] * z[i] * r[i];
      rr += r[i] * r[i];
    }
    const double beta = rz_new / rz;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] * r[i] + beta * p[i];
    rz = rz_new;
    rn = sqrt(rr);
    ++it;
  }
  *rel = rn / fn;
  return it;
}
