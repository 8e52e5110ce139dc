// Optimisation-step launchers and the device state of the OC search for lambda.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace amr {

struct DeviceMesh;

// Device state of the OC search (one per context): the target volume and tolerance (set by the
// host), the bracket on s = lambda^-eta, the next candidates, and the result.
struct OcState {
  double l1, l2, target, tol;   // final lambda bracket [l1, l2]; target volume; relative tolerance
  double change, lambda;        // max |rho_new - rho| and the lambda used
  int done, iters;              // search finished; search launches that did work
  double s_lo, s_hi;            // bracket on s (s_hi = +inf while unbounded)
  double c0, c1;                // candidates of the next launch (c1 <= 0: none)
  double step;                  // the last accepted Newton step (for the halving safeguard)
};

cudaError_t launch_sensitivity(const DeviceMesh &m, const double *rho, const double *uf, double *dc,
                               double *partials, unsigned int *ticket, double *compliance, cudaStream_t s);
cudaError_t launch_filter(const DeviceMesh &m, const double *rho, const double *x, double rmin, int mode,
                          double *out, cudaStream_t s);
// tab: Ne entries of scratch (the lambda-free factor, the bounds and the volume per element).
// The OC update is three launchers on one stream: the table and the first candidate, `steps`
// search launches (each returns at once after the search has finished), and the new densities
// with the largest change.
cudaError_t launch_oc_init(const DeviceMesh &m, const double *rho, const double *dc, double eta, double move,
                           double rmin, double4_32a *tab, double *partials, unsigned int *ticket, OcState *st,
                           cudaStream_t s);
cudaError_t launch_oc_search(const DeviceMesh &m, double eta, const double4_32a *tab, double *partials,
                             unsigned int *ticket, OcState *st, int steps, cudaStream_t s);
cudaError_t launch_oc_final(const DeviceMesh &m, const double *rho, double eta, const double4_32a *tab,
                            double *rho_new, double *partials, unsigned int *ticket, OcState *st, cudaStream_t s);

}  // namespace amr
