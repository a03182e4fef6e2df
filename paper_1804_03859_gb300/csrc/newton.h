// Internal interface of the Newton-Krylov driver (not part of the C ABI).
#pragma once

#include "stepper.cuh"

namespace nsstab {

// q: device n-vector, in/out.  st: nonlinear map and residual.  Jacobian
// products: tan->tangent (exact discrete tangent; tan a two-member stepper)
// when tan is not null, else lin->step_linear about q (frozen base; lin may
// be st).  All on the same grid and stream.
int newton_run(StepperBase* st, StepperBase* lin, StepperBase* tan, cudaStream_t stream, long n, double* q,
               int nsteps, int m, double gmres_rtol, int max_restarts, double tol, int max_newton, double* res_out,
               int* iters_out, int* mv_out);

}  // namespace nsstab
