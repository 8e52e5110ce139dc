// Optimisation-step launchers and the device state of the OC bisection.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace amr {

struct DeviceMesh;

struct OcState {
  double l1, l2, target, tol;
  double change, lambda;
  int done, iters;
};

cudaError_t launch_sensitivity(const DeviceMesh &m, const double *rho, const double *uf, double *dc,
                               double *partials, unsigned int *ticket, double *compliance, cudaStream_t s);
cudaError_t launch_filter(const DeviceMesh &m, const double *rho, const double *x, double rmin, int mode,
                          double *out, cudaStream_t s);
cudaError_t launch_oc(const DeviceMesh &m, const double *rho, const double *dc, double eta, double move, double rmin,
                      double *rho_new, double *partials, unsigned int *ticket, OcState *st, int max_bisect,
                      cudaStream_t s);

}  // namespace amr
