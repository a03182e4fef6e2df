// Internal interface of the Krylov eigen-driver (not part of the C ABI).
#pragma once

#include <complex>
#include <functional>
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

// The same driver over nb members of possibly different lengths nm[b]
// (device vectors on `stream`): prod(in, out) applies each member's M to
// in[b] into out[b] for every non-null in[b] (null: the member is finished
// and is skipped).
int arnoldi_members_run(const std::function<int(const double* const*, double* const*)>& prod, int nb,
                        const long* nm, cudaStream_t stream, const double* const* v0, int m, int nev, double tol,
                        int max_restarts, std::vector<ArnoldiOut>& outs);

// Block Krylov-Schur: one eigenproblem per parameter set of the stepper,
// each with a block of b = members / sets vectors per product with M (the b
// members of a set share its base flow), all sets in lockstep rounds.
// v0: host array of `members` device pointers (set s's start block is
// v0[s b .. s b + b - 1], linearly independent); outs[s] receives set s's
// results.  Requires m >= 2 (nev + 1) + 2 b.
int block_arnoldi_run(StepperBase* st, cudaStream_t stream, long n, const double* const* v0, int m, int nev,
                      double tol, int max_restarts, int nsteps, std::vector<ArnoldiOut>& outs);

}  // namespace nsstab
