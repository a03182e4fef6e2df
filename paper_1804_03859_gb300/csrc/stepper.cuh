// Internal interface of the time-stepper (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace nsstab {

// Precision-independent face of a stepper; StepperImpl<T> implements it for
// T = double (FP64 stepper) and T = float (FP32 stepper with FP64 I/O).
//
// A stepper advances a batch of B = S * per_set members on one grid: member
// m belongs to parameter set m / per_set (its own Reynolds number and
// cylinder diameter, and its own base flow for the linearised step).  Field
// arguments are [B][ny][nx] (base flows [S][ny][nx]); a single stepper is
// the batch B = S = 1.
struct StepperBase {
    virtual ~StepperBase() {}
    virtual int init() = 0;
    virtual int members() const = 0;
    virtual int sets() const = 0;
    virtual int poisson(const double* omega, double* psi) = 0;
    virtual int step_nonlinear(double* omega, int nsteps) = 0;
    virtual int set_base(const double* base_omega) = 0;
    // base flows by pointer: host array of S device pointers
    virtual int set_base_ptrs(const double* const* base_omegas) = 0;
    virtual int step_linear(const double* v_in, double* v_out, int nsteps) = 0;
    // per-member device pointers (host arrays of B); a null input pointer
    // leaves that member out of this call
    virtual int step_linear_ptrs(const double* const* in, double* const* out, int nsteps) = 0;
    // exact discrete tangent of Phi_T (nsteps nonlinear steps) at q applied
    // to v_in, by co-integration; needs a batch of two members, one set
    virtual int tangent(const double* q, const double* v_in, double* v_out, int nsteps) = 0;
    virtual int residual(const double* q, double* r) = 0;   // r: host [B]
    virtual int sfd(double* omega, double chi, double Delta, double tol, long max_steps,
                    int check_every, double* r, long* steps) = 0;
    virtual int launches_per_step() const = 0;
    // time each kernel of `nsteps` linearised steps from v with CUDA events
    // on the stepper's stream; ms[k] accumulates kernel k (kNumStepKernels)
    virtual int profile_linear(const double* v, int nsteps, double* ms) = 0;
    // time every valid launch configuration of each step kernel and keep the
    // fastest; chosen[2k], chosen[2k+1] = (log2 elements per thread, sequences per block)
    virtual int autotune(int reps, int* chosen) = 0;
    virtual int plan_of(int kid, int* le, int* per) const = 0;
    virtual int set_plan(int kid, int le, int per) = 0;
    // FP32 steppers: run the two row passes of a step as fused kernels over
    // strips of R rows (rowroll.cuh); R = 0 returns to the six-kernel step
    virtual int set_fused_rows(int R) = 0;
    virtual int fused_rows() const = 0;
};

// Independent solves on grids of different sizes, advanced together by one
// persistent launch per step kernel (FP32; ragged.cuh).  add_group adds k
// solves on one grid (nsteps = T/dt steps per product with M) with their
// base flows; finalize fixes the launch plans and captures a product round;
// product applies every member's M (members numbered group by group; a null
// in[m] skips member m).
struct RaggedBase {
    virtual ~RaggedBase() {}
    virtual int add_group(const nsstab_config& cfg, int k, const double* Re, const double* D, int nsteps,
                          const double* const* bases) = 0;
    virtual int finalize() = 0;
    virtual int members() const = 0;
    virtual int groups() const = 0;
    virtual long n_of(int m) const = 0;
    virtual int product(const double* const* in, double* const* out) = 0;
    virtual int launches_per_round() const = 0;
};
RaggedBase* make_ragged_f32(cudaStream_t stream);
constexpr int kRagMaxGroups = 8;   // grids per ragged launch

constexpr int kNumStepKernels = 6;   // col_poisson, row_inverse(psi), row_forward(rhs),
                                     // col_update, row_inverse(omega*, psi*), row_forward(pen)
StepperBase* make_stepper(const nsstab_config& cfg, int nsets, const double* Re, const double* D, int per_set,
                          cudaStream_t stream);
int validate_config(const nsstab_config& cfg);

// Krylov helpers (krylov_kernels.cu), all FP64 on `stream`.
struct GsWork {
    double* partial = nullptr;   // [grid][max_cols]
    double* hdev = nullptr;      // [2][max_cols]
    double* hhost = nullptr;     // pinned [2*max_cols + 2]
    int grid = 0;
    int max_cols = 0;
    int alloc(int max_cols_);
    void release();
};
int cgs2(const double* V, long ldv, long n, int j, double* w, double* h, double* beta,
         GsWork& ws, cudaStream_t stream);

// Workspace of the batched Gram-Schmidt kernels (one member per grid.y).
struct GsBatch {
    double* partial = nullptr;   // [B][grid][max_cols]
    double* hdev = nullptr;      // h1, h2, beta^2: [3][B][max_cols]
    double* hhost = nullptr;     // pinned copy of hdev
    double* sdev = nullptr;      // [B] scale factors
    int* jdev = nullptr;         // [2][B] column counts
    long* ndev = nullptr;        // [B] member lengths (members of different grids)
    double** ptrs = nullptr;     // [2][B] member pointers
    int B = 0, max_cols = 0, grid = 0;
    int alloc(int nmem, int cols);
    void release();
};
// nm (host, optional): per-member lengths, each also its basis's leading
// dimension, in place of n and ldv (members on grids of different sizes).
int cgs2_batch(int nmem, const double* const* V, long ldv, long n, const int* j, double* const* w,
               double* h, int ldh, double* beta, GsBatch& ws, cudaStream_t stream, const long* nm = nullptr);
int scale_batch(int nmem, double* const* w, long n, const double* s, GsBatch& ws, cudaStream_t stream,
                const long* nm = nullptr);
// Blocked Gram-Schmidt (two passes) of the b <= kMaxGsBlock columns of W[s]
// (ldw apart) against the first J[s] columns of V[s], for every set with
// J[s] > 0: H = V^T W, W -= V H, twice, each a single read of V for all b
// columns.  H[s][c * b + q] (host, row stride ldh) = the summed coefficients
// of both passes.  The columns of W are not made orthogonal to each other.
constexpr int kMaxGsBlock = 8;
int bcgs2_batch(int S, const double* const* V, long ldv, long n, const int* J, double* const* W, long ldw, int b,
                double* H, int ldh, GsBatch& ws, cudaStream_t stream);
int vec_norm(const double* x, long n, double* out, GsWork& ws, cudaStream_t stream);
int vec_scale(double* dst, const double* src, long n, double s, cudaStream_t stream);
int vec_axpby(double* dst, double a, const double* x, double b, const double* y, long n, cudaStream_t stream);
// out[:, c] = sum_k V[:, k] C[k, c] for c < p (C: device, column-major
// m x p); out must not alias V.
int basis_combine(const double* V, long ldv, long n, int m, const double* C_dev, int p,
                  double* out, long ldo, cudaStream_t stream);

}  // namespace nsstab
