// Internal interface of the Krylov eigen-driver (not part of the C ABI).
#pragma once

#include <complex>
#include <vector>

#include "stepper.cuh"

namespace nsstab {

struct ArnoldiOut {
    std::vector<std::complex<double>> mu;   // leading Ritz values
    std::vector<double> resid;              // |b^T y| of each
    double* eigvecs = nullptr;              // device [k][n] or null
    int n_eig = 0, n_conv = 0, n_matvec = 0, restarts = 0;
    int status = NSSTAB_OK;
    double done_at = 0.0;                   // steady-clock seconds when the member finished
};

// Seconds on the steady clock (the time base of ArnoldiOut::done_at).
double steady_seconds();

// One eigenproblem per member of the stepper's batch.  v0: host array of
// `members` device pointers, each n values; nsteps = T/dt linearised steps
// per product with M; outs[b] receives member b's results (set
// outs[b].eigvecs before the call to get Ritz vectors).
int arnoldi_batch_run(StepperBase* st, cudaStream_t stream, long n, const double* const* v0, int m, int nev,
                      double tol, int max_restarts, int nsteps, std::vector<ArnoldiOut>& outs);

// One eigenproblem solved with a block of b = st->members() vectors per
// product with M (block Krylov-Schur); the members must share one base flow
// (one parameter set).  v0: host array of b device pointers (the start
// block, linearly independent).  Requires m >= 2 (nev + 1) + 2 b.
int block_arnoldi_run(StepperBase* st, cudaStream_t stream, long n, const double* const* v0, int m, int nev,
                      double tol, int max_restarts, int nsteps, ArnoldiOut& out);

}  // namespace nsstab
