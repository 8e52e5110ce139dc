// Device-resident scalars of one CG run and the vector-kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace amr {

struct SolveScalars {
  double rz, pq, alpha, beta;
  double rr, rr0;          // current / initial ||r||^2 of this CG run
  double stop_ratio2;      // stop when rr <= max(stop_ratio2 * rr0, stop_abs_rr)
  double stop_abs_rr;
  double stop_rr;
  double scratch[7];
  int it, max_it, done, nonfinite, last_beta_skipped, pad[3];
};

int vec_grid(int64_t n);
template <typename TX, typename T>
cudaError_t launch_update(TX *x, const T *p, const T *q, T *r, const T *dinv, int64_t n, SolveScalars *sc,
                          double *partials, unsigned int *ticket, cudaStream_t s);
template <typename TX, typename T>
cudaError_t launch_update_nodes(TX *x, const T *p, const T *q, T *r, const T *dinv, int64_t Nn,
                                const int32_t *sh_of_node, const int32_t *sh_ptr, const T *part, SolveScalars *sc,
                                double *partials, unsigned int *ticket, cudaStream_t s);
template <typename T>
cudaError_t launch_pupdate(T *p, const T *r, const T *dinv, int64_t n, SolveScalars *sc, cudaStream_t s);
template <typename T>
cudaError_t launch_start(const double *f, const double *q, double scale, T *r, T *p, const T *dinv, int64_t n,
                         SolveScalars *sc, double *partials, unsigned int *ticket, cudaStream_t s);
cudaError_t launch_residual64(const double *f, const double *q, double *r, int64_t n, double *out,
                              double *partials, unsigned int *ticket, cudaStream_t s);
cudaError_t launch_correct(double *u, float *d, double scale, int64_t n, cudaStream_t s);
cudaError_t launch_mask(const uint8_t *nflag, double *u, int64_t Nn, cudaStream_t s);

}  // namespace amr
