// Device-resident scalars of one CG run and the vector-kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace amr {

struct SolveScalars {
  double rz, pq, alpha, beta;
  double rr, rr0;          // current / initial ||r||^2 of this CG run
  double stop_ratio2;      // stop when rr <= max(stop_ratio2 * rrmax, stop_abs_rr)
  double stop_abs_rr;
  double stop_rr;
  double rrmax;            // largest ||r||^2 since the run (or the last residual replacement) began
  double rz_prev;          // rz of the previous iteration (the one p was built from)
  double rp;               // r^T p after a residual replacement
  double scratch[4];
  int it, max_it, done, nonfinite, last_beta_skipped, pad[3];
};

int vec_grid(int64_t n);
template <typename TX, typename T>
cudaError_t launch_update(TX *x, const T *p, const T *q, T *r, const T *dinv, int64_t n, SolveScalars *sc,
                          double *partials, unsigned int *ticket, cudaStream_t s);
template <typename TX, typename T>
cudaError_t launch_update_nodes(TX *x, const T *p, const T *q, T *r, const T *dinv, int64_t Nn,
                                const int32_t *sh_of_node, const int32_t *sh_ptr, const T *part, SolveScalars *sc,
                                double *partials, unsigned int *ticket, cudaStream_t s, bool twolevel = false);
// The FP32 update for nv load cases in one launch (grid y = case): vectors vst apart, shared-node
// partials pst apart, scalars sc[case], reduction partials 2 * grid apart, tickets[case].
cudaError_t launch_update_nodes_cases(int nv, float *x, const float *p, const float *q, float *r, int64_t vst,
                                      const float *dinv, int64_t Nn, const int32_t *sh_of_node, const int32_t *sh_ptr,
                                      const float *part, int64_t pst, SolveScalars *sc, double *partials,
                                      unsigned int *tickets, cudaStream_t s, bool twolevel);
template <typename T>
cudaError_t launch_pupdate(T *p, const T *r, const T *dinv, int64_t n, SolveScalars *sc, cudaStream_t s);
template <typename T>
cudaError_t launch_start(const double *f, const double *q, double scale, T *r, T *p, const T *dinv, int64_t n,
                         SolveScalars *sc, double *partials, unsigned int *ticket, cudaStream_t s);
cudaError_t launch_residual64(const double *f, const double *q, double *r, int64_t n, double *out,
                              double *partials, unsigned int *ticket, cudaStream_t s);
cudaError_t launch_correct(double *u, float *d, double scale, int64_t n, cudaStream_t s);
// Residual replacement of the mixed solver: r = scale * r64 (the FP64 true residual),
// p *= c (the previous run's units to the new ones), then p made orthogonal to r
// within span{Dinv r} and p = Dinv r + beta p; CG then continues with the kept direction.
// dots_only: stop after the dot products (the two-level preconditioner builds p itself).
cudaError_t launch_replace(const double *r64, double scale, double c, float *r, float *p, const float *dinv,
                           int64_t n, double stop_abs_rr, int max_it, SolveScalars *sc, double *partials,
                           unsigned int *ticket, cudaStream_t s, bool dots_only = false);
cudaError_t launch_mask(const uint8_t *nflag, double *u, int64_t Nn, cudaStream_t s);

}  // namespace amr
