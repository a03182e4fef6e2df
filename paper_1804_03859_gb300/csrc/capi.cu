// extern "C" entry points of libnsstab.so (declared in include/nsstab.h):
// argument checking, the stepper handle, and dispatch to the stepper
// (stepper.cu), the Krylov driver (arnoldi.cu) and the Krylov kernels
// (krylov.cu).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "arnoldi.h"
#include "dense_eig.h"
#include "newton.h"
#include "stepper.cuh"

struct nsstab_stepper {
    nsstab_config cfg;
    cudaStream_t stream;
    nsstab::StepperBase* impl;
    nsstab::GsWork gs;
    bool have_base;
};

namespace nsstab {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

static int bad_arg(const char* msg) {
    set_error(msg);
    return NSSTAB_ERR_INVALID_ARG;
}

static int steps_for(const nsstab_config& cfg, double T, int* nsteps) {
    const double ns = T / cfg.dt;
    const double k = std::round(ns);
    if (!(T > 0) || k < 1 || std::fabs(ns - k) > 1e-9 * std::max(1.0, ns) || k > 1e9)
        return bad_arg("T must be a positive whole number of time steps");
    *nsteps = (int)k;
    return NSSTAB_OK;
}

}  // namespace nsstab

using namespace nsstab;

extern "C" {

void nsstab_config_default(nsstab_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->nx = 128;
    c->ny = 64;
    c->Lx = 16.0;
    c->Ly = 8.0;
    c->dt = 0.01;
    c->Re = 50.0;
    c->Uinf = 1.0;
    c->cyl_x = 4.0;
    c->cyl_y = 4.0;
    c->cyl_D = 1.0;
    c->eta = 1e-3;
    c->mask_cells = 2.0;
    c->sponge_frac = 0.1;
    c->sponge_sigma = 10.0;
    c->precision = 64;
}

const char* nsstab_last_error(void) { return last_error(); }

static int create_impl(const nsstab_config* cfg, int nsets, const double* Re, const double* D, int per_set,
                       void* stream, nsstab_stepper** out) {
    NS_TRY(validate_config(*cfg));
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        set_error("stepper_create: no CUDA device");
        return NSSTAB_ERR_CUDA;
    }
    nsstab_stepper* st = new nsstab_stepper();
    st->cfg = *cfg;
    st->stream = (cudaStream_t)stream;
    st->have_base = false;
    st->impl = make_stepper(*cfg, nsets, Re, D, per_set, st->stream);
    const int rc = st->impl->init();
    if (rc != NSSTAB_OK) {
        delete st->impl;
        delete st;
        return rc;
    }
    *out = st;
    return NSSTAB_OK;
}

int stepper_create(const nsstab_config* cfg, void* stream, nsstab_stepper** out) {
    if (!cfg || !out) return bad_arg("stepper_create: null argument");
    *out = nullptr;
    return create_impl(cfg, 1, nullptr, nullptr, 1, stream, out);
}

int batch_create(const nsstab_config* cfg, int nsets, const double* Re, const double* cyl_D, int per_set,
                 void* stream, nsstab_stepper** out) {
    if (!cfg || !out) return bad_arg("batch_create: null argument");
    *out = nullptr;
    if (nsets < 1 || per_set < 1 || (long)nsets * per_set > 65535)
        return bad_arg("batch_create: need nsets >= 1, per_set >= 1, nsets * per_set <= 65535");
    for (int k = 0; k < nsets; ++k) {
        if (Re && !(Re[k] > 0)) return bad_arg("batch_create: every Re must be positive");
        if (cyl_D && !(cyl_D[k] >= 0)) return bad_arg("batch_create: every cyl_D must be >= 0");
    }
    return create_impl(cfg, nsets, Re, cyl_D, per_set, stream, out);
}

int stepper_members(nsstab_stepper* st, int* members, int* sets) {
    if (!st || !members || !sets) return bad_arg("stepper_members: null argument");
    *members = st->impl->members();
    *sets = st->impl->sets();
    return NSSTAB_OK;
}

void stepper_destroy(nsstab_stepper* st) {
    if (!st) return;
    cudaStreamSynchronize(st->stream);
    st->gs.release();
    delete st->impl;
    delete st;
}

int stepper_poisson(nsstab_stepper* st, const double* omega, double* psi) {
    if (!st || !omega || !psi) return bad_arg("stepper_poisson: null argument");
    return st->impl->poisson(omega, psi);
}

int step_nonlinear(nsstab_stepper* st, double* omega, int nsteps) {
    if (!st || !omega) return bad_arg("step_nonlinear: null argument");
    if (nsteps < 0) return bad_arg("step_nonlinear: nsteps < 0");
    return st->impl->step_nonlinear(omega, nsteps);
}

int stepper_set_base(nsstab_stepper* st, const double* base_omega) {
    if (!st || !base_omega) return bad_arg("stepper_set_base: null argument");
    NS_TRY(st->impl->set_base(base_omega));
    st->have_base = true;
    return NSSTAB_OK;
}

int apply_expTL(nsstab_stepper* st, const double* base_omega, const double* v_in, double* v_out, double T) {
    if (!st || !v_in || !v_out) return bad_arg("apply_expTL: null argument");
    int nsteps = 0;
    NS_TRY(steps_for(st->cfg, T, &nsteps));
    if (base_omega) {
        NS_TRY(st->impl->set_base(base_omega));
        st->have_base = true;
    } else if (!st->have_base) {
        return bad_arg("apply_expTL: no base flow (pass base_omega or call stepper_set_base)");
    }
    return st->impl->step_linear(v_in, v_out, nsteps);
}

int stepper_residual(nsstab_stepper* st, const double* q, double* r) {
    if (!st || !q || !r) return bad_arg("stepper_residual: null argument");
    NS_TRY(st->impl->residual(q, r));
    for (int m = 0; m < st->impl->members(); ++m)
        if (!std::isfinite(r[m])) return NSSTAB_DIVERGED;
    return NSSTAB_OK;
}

int sfd_baseflow(nsstab_stepper* st, double* omega, double chi, double Delta, double tol, long max_steps,
                 int check_every, double* residual, long* steps) {
    if (!st || !omega || !residual || !steps) return bad_arg("sfd_baseflow: null argument");
    if (!(chi >= 0) || !(Delta > 0) || !(tol >= 0) || max_steps < 1 || check_every < 1)
        return bad_arg("sfd_baseflow: need chi >= 0, Delta > 0, tol >= 0, max_steps >= 1, check_every >= 1");
    return st->impl->sfd(omega, chi, Delta, tol, max_steps, check_every, residual, steps);
}

int arnoldi_eigs(nsstab_stepper* st, const double* base_omega, const double* v0, int m, int nev, double tol,
                 int max_restarts, double T, double* eig_re, double* eig_im, double* resid, double* eigvecs,
                 int* n_eig, int* n_conv, int* n_matvec) {
    if (!st || !v0 || !eig_re || !eig_im || !resid || !n_eig || !n_conv || !n_matvec)
        return bad_arg("arnoldi_eigs: null argument");
    if (st->impl->members() != 1) return bad_arg("arnoldi_eigs: single steppers only (use batch_arnoldi_eigs)");
    const long n = (long)st->cfg.nx * st->cfg.ny;
    if (m < 2 || m > 1024 || m >= n) return bad_arg("arnoldi_eigs: need 2 <= m <= min(nx*ny - 1, 1024)");
    if (nev < 1 || nev >= m) return bad_arg("arnoldi_eigs: need 1 <= nev < m");
    if (max_restarts < 0) return bad_arg("arnoldi_eigs: max_restarts < 0");
    if (!(tol >= 0)) return bad_arg("arnoldi_eigs: tol < 0");
    int nsteps = 0;
    NS_TRY(steps_for(st->cfg, T, &nsteps));
    if (base_omega) {
        NS_TRY(st->impl->set_base(base_omega));
        st->have_base = true;
    } else if (!st->have_base) {
        return bad_arg("arnoldi_eigs: no base flow (pass base_omega or call stepper_set_base)");
    }
    std::vector<ArnoldiOut> outs(1);
    outs[0].eigvecs = eigvecs;
    const double* v0p[1] = {v0};
    const int rc = arnoldi_batch_run(st->impl, st->stream, n, v0p, m, nev, tol, max_restarts, nsteps, outs);
    if (rc < 0) return rc;
    const ArnoldiOut& out = outs[0];
    for (int s = 0; s < out.n_eig; ++s) {
        eig_re[s] = out.mu[s].real();
        eig_im[s] = out.mu[s].imag();
        resid[s] = out.resid[s];
    }
    *n_eig = out.n_eig;
    *n_conv = out.n_conv;
    *n_matvec = out.n_matvec;
    return rc != NSSTAB_OK ? rc : out.status;
}

int batch_arnoldi_eigs(nsstab_stepper* st, const double* base_omegas, const double* v0, int m, int nev, double tol,
                       int max_restarts, double T, double* eig_re, double* eig_im, double* resid, double* eigvecs,
                       int* n_eig, int* n_conv, int* n_matvec) {
    if (!st || !v0 || !eig_re || !eig_im || !resid || !n_eig || !n_conv || !n_matvec)
        return bad_arg("batch_arnoldi_eigs: null argument");
    const long n = (long)st->cfg.nx * st->cfg.ny;
    if (m < 2 || m > 1024 || m >= n) return bad_arg("batch_arnoldi_eigs: need 2 <= m <= min(nx*ny - 1, 1024)");
    if (nev < 1 || nev >= m) return bad_arg("batch_arnoldi_eigs: need 1 <= nev < m");
    if (max_restarts < 0) return bad_arg("batch_arnoldi_eigs: max_restarts < 0");
    if (!(tol >= 0)) return bad_arg("batch_arnoldi_eigs: tol < 0");
    int nsteps = 0;
    NS_TRY(steps_for(st->cfg, T, &nsteps));
    if (base_omegas) {
        NS_TRY(st->impl->set_base(base_omegas));
        st->have_base = true;
    } else if (!st->have_base) {
        return bad_arg("batch_arnoldi_eigs: no base flows (pass base_omegas or call stepper_set_base)");
    }
    const int B = st->impl->members();
    std::vector<ArnoldiOut> outs(B);
    if (eigvecs)
        for (int b = 0; b < B; ++b) outs[b].eigvecs = eigvecs + (size_t)b * (nev + 1) * n;
    std::vector<const double*> v0p(B);
    for (int b = 0; b < B; ++b) v0p[b] = v0 + (size_t)b * n;
    const int rc = arnoldi_batch_run(st->impl, st->stream, n, v0p.data(), m, nev, tol, max_restarts, nsteps, outs);
    if (rc < 0) return rc;
    int status = rc;
    for (int b = 0; b < B; ++b) {
        const ArnoldiOut& o = outs[b];
        for (int s = 0; s < o.n_eig; ++s) {
            eig_re[(size_t)b * (nev + 1) + s] = o.mu[s].real();
            eig_im[(size_t)b * (nev + 1) + s] = o.mu[s].imag();
            resid[(size_t)b * (nev + 1) + s] = o.resid[s];
        }
        n_eig[b] = o.n_eig;
        n_conv[b] = o.n_conv;
        n_matvec[b] = o.n_matvec;
        if (status == NSSTAB_OK && o.status != NSSTAB_OK) status = o.status;
    }
    return status;
}

int block_arnoldi_eigs(nsstab_stepper* st, const double* base_omega, const double* v0, int m, int nev, double tol,
                       int max_restarts, double T, double* eig_re, double* eig_im, double* resid, double* eigvecs,
                       int* n_eig, int* n_conv, int* n_matvec) {
    if (!st || !v0 || !eig_re || !eig_im || !resid || !n_eig || !n_conv || !n_matvec)
        return bad_arg("block_arnoldi_eigs: null argument");
    const int S = st->impl->sets();
    const int b = st->impl->members() / S;
    const long n = (long)st->cfg.nx * st->cfg.ny;
    if (nev < 1) return bad_arg("block_arnoldi_eigs: need nev >= 1");
    if (m > 1024 || m + 2L * b >= n || m < 2 * (nev + 1) + 2 * b)
        return bad_arg("block_arnoldi_eigs: need 2 (nev + 1) + 2 b <= m <= 1024 and m + 2 b < nx*ny");
    // blocked Gram-Schmidt: at most kMaxGsBlock columns a block, and the
    // (m + b) x b coefficients of a pass in the default 48 KB of shared memory
    if (b > kMaxGsBlock || (long)(m + b) * b > 6144)
        return bad_arg("block_arnoldi_eigs: need b <= 8 and (m + b) b <= 6144 (blocked Gram-Schmidt)");
    if (max_restarts < 0) return bad_arg("block_arnoldi_eigs: max_restarts < 0");
    if (!(tol >= 0)) return bad_arg("block_arnoldi_eigs: tol < 0");
    int nsteps = 0;
    NS_TRY(steps_for(st->cfg, T, &nsteps));
    if (base_omega) {
        NS_TRY(st->impl->set_base(base_omega));
        st->have_base = true;
    } else if (!st->have_base) {
        return bad_arg("block_arnoldi_eigs: no base flow (pass base_omega or call stepper_set_base)");
    }
    std::vector<const double*> v0p((size_t)S * b);
    for (size_t i = 0; i < v0p.size(); ++i) v0p[i] = v0 + i * n;
    std::vector<ArnoldiOut> outs(S);
    if (eigvecs)
        for (int s = 0; s < S; ++s) outs[s].eigvecs = eigvecs + (size_t)s * (nev + 1) * n;
    const int rc = block_arnoldi_run(st->impl, st->stream, n, v0p.data(), m, nev, tol, max_restarts, nsteps, outs);
    if (rc < 0) return rc;
    int status = rc;
    for (int s = 0; s < S; ++s) {
        const ArnoldiOut& o = outs[s];
        for (int q = 0; q < o.n_eig; ++q) {
            eig_re[(size_t)s * (nev + 1) + q] = o.mu[q].real();
            eig_im[(size_t)s * (nev + 1) + q] = o.mu[q].imag();
            resid[(size_t)s * (nev + 1) + q] = o.resid[q];
        }
        n_eig[s] = o.n_eig;
        n_conv[s] = o.n_conv;
        n_matvec[s] = o.n_matvec;
        if (status == NSSTAB_OK && o.status != NSSTAB_OK) status = o.status;
    }
    return status;
}

int apply_tangent(nsstab_stepper* st, const double* q, const double* v_in, double* v_out, double T) {
    if (!st || !q || !v_in || !v_out) return bad_arg("apply_tangent: null argument");
    if (st->impl->members() != 2 || st->impl->sets() != 1)
        return bad_arg("apply_tangent: needs a batch of two members and one parameter set");
    int nsteps = 0;
    NS_TRY(steps_for(st->cfg, T, &nsteps));
    st->have_base = false;
    return st->impl->tangent(q, v_in, v_out, nsteps);
}

int newton_krylov_fixedpoint_ex(nsstab_stepper* st, nsstab_stepper* lin_st, double* omega, double T, int gmres_m,
                                double gmres_rtol, int gmres_restarts, double tol, int max_newton, int jacobian,
                                double* residual, int* newton_iters, int* matvecs) {
    if (!st || !omega || !residual || !newton_iters || !matvecs)
        return bad_arg("newton_krylov_fixedpoint: null argument");
    if (jacobian != NSSTAB_JACOBIAN_TANGENT && jacobian != NSSTAB_JACOBIAN_FROZEN)
        return bad_arg("newton_krylov_fixedpoint: jacobian must be NSSTAB_JACOBIAN_TANGENT or _FROZEN");
    nsstab_stepper* lin = lin_st ? lin_st : st;
    if (st->impl->members() != 1 || lin->impl->members() != 1)
        return bad_arg("newton_krylov_fixedpoint: single steppers only");
    if (lin->cfg.nx != st->cfg.nx || lin->cfg.ny != st->cfg.ny || lin->cfg.dt != st->cfg.dt)
        return bad_arg("newton_krylov_fixedpoint: lin_st must have the grid and dt of st");
    if (gmres_m < 1 || gmres_m > 1024 || gmres_restarts < 0 || !(gmres_rtol > 0) || !(tol >= 0) || max_newton < 0)
        return bad_arg("newton_krylov_fixedpoint: need 1 <= gmres_m <= 1024, gmres_restarts >= 0, gmres_rtol > 0, "
                       "tol >= 0, max_newton >= 0");
    int nsteps = 0;
    NS_TRY(steps_for(st->cfg, T, &nsteps));
    const long n = (long)st->cfg.nx * st->cfg.ny;
    StepperBase* tan = nullptr;
    if (jacobian == NSSTAB_JACOBIAN_TANGENT) {
        // the two-member stepper of the co-integration, in lin's arithmetic, on st's stream
        tan = make_stepper(lin->cfg, 1, &lin->cfg.Re, &lin->cfg.cyl_D, 2, st->stream);
        const int ri = tan->init();
        if (ri != NSSTAB_OK) {
            delete tan;
            return ri;
        }
    }
    const int rc = newton_run(st->impl, lin->impl, tan, st->stream, n, omega, nsteps, gmres_m, gmres_rtol,
                              gmres_restarts, tol, max_newton, residual, newton_iters, matvecs);
    if (tan) {
        delete tan;
    } else {
        lin->have_base = true;   // lin now holds the last iterate as its base
    }
    return rc;
}

int newton_krylov_fixedpoint(nsstab_stepper* st, double* omega, double T, int gmres_m, double tol, int max_newton,
                             double* residual, int* newton_iters, int* matvecs) {
    return newton_krylov_fixedpoint_ex(st, nullptr, omega, T, gmres_m, 1e-3, 2, tol, max_newton,
                                       NSSTAB_JACOBIAN_TANGENT, residual, newton_iters, matvecs);
}

int stepper_profile_linear(nsstab_stepper* st, const double* v, int nsteps, double* kernel_ms) {
    if (!st || !v || !kernel_ms || nsteps < 1) return bad_arg("stepper_profile_linear: bad argument");
    if (!st->have_base) return bad_arg("stepper_profile_linear: no base flow set");
    return st->impl->profile_linear(v, nsteps, kernel_ms);
}

int stepper_autotune(nsstab_stepper* st, int reps, int* plans) {
    if (!st || reps < 1 || reps > 1000) return bad_arg("stepper_autotune: bad argument");
    return st->impl->autotune(reps, plans);
}

int stepper_set_plan(nsstab_stepper* st, int kernel, int log2_elems, int per_block) {
    if (!st) return bad_arg("stepper_set_plan: null stepper");
    return st->impl->set_plan(kernel, log2_elems, per_block);
}

int stepper_get_plan(nsstab_stepper* st, int kernel, int* log2_elems, int* per_block) {
    if (!st || !log2_elems || !per_block) return bad_arg("stepper_get_plan: null argument");
    const int rc = st->impl->plan_of(kernel, log2_elems, per_block);
    if (rc != NSSTAB_OK) return bad_arg("stepper_get_plan: kernel must be in [0, 6)");
    return NSSTAB_OK;
}

int stepper_set_fused_rows(nsstab_stepper* st, int rows_per_strip) {
    if (!st) return bad_arg("stepper_set_fused_rows: null stepper");
    if (rows_per_strip < 0) return bad_arg("stepper_set_fused_rows: rows_per_strip must be >= 0");
    const int rc = st->impl->set_fused_rows(rows_per_strip);
    if (rc == NSSTAB_OK) cudaStreamSynchronize(st->stream);
    return rc;
}

int stepper_get_fused_rows(nsstab_stepper* st, int* rows_per_strip) {
    if (!st || !rows_per_strip) return bad_arg("stepper_get_fused_rows: null argument");
    *rows_per_strip = st->impl->fused_rows();
    return NSSTAB_OK;
}

int cgs2_orthogonalize(const double* V, long ldv, long n, int j, double* w, double* h, double* beta, void* stream) {
    if (!w || !beta || (j > 0 && (!V || !h))) return bad_arg("cgs2_orthogonalize: null argument");
    if (n < 1 || j < 0 || j > 4096 || (j > 0 && ldv < n)) return bad_arg("cgs2_orthogonalize: bad sizes");
    static thread_local GsWork ws;   // grown on demand, kept for the thread's lifetime
    return cgs2(V, ldv, n, j, w, h, beta, ws, (cudaStream_t)stream);
}

int nsstab_dense_eig(int n, const double* A, int is_hessenberg, double* wr, double* wi, double* vr, double* vi) {
    if (n < 1 || !A || !wr || !wi) return bad_arg("nsstab_dense_eig: bad argument");
    std::vector<double> T(A, A + (size_t)n * n), Z((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Z[i + (size_t)i * n] = 1.0;
    if (!is_hessenberg) dense::hessenberg(n, T.data(), Z.data());
    if (dense::schur(n, T.data(), Z.data()) != 0) {
        set_error("nsstab_dense_eig: QR iteration did not converge");
        return NSSTAB_ERR_NUMERICAL;
    }
    const std::vector<dense::cd> ev = dense::schur_eigenvalues(n, T.data());
    for (int i = 0; i < n; ++i) {
        wr[i] = ev[i].real();
        wi[i] = ev[i].imag();
    }
    if (vr && vi) {
        for (int i = 0; i < n; ++i) {
            std::vector<dense::cd> y;
            if (i > 0 && T[i + (size_t)(i - 1) * n] != 0.0) {
                y = dense::schur_eigenvector(n, T.data(), Z.data(), i - 1, ev[i - 1]);
                for (auto& v : y) v = std::conj(v);
            } else {
                y = dense::schur_eigenvector(n, T.data(), Z.data(), i, ev[i]);
            }
            for (int r = 0; r < n; ++r) {
                vr[r + (size_t)i * n] = y[r].real();
                vi[r + (size_t)i * n] = y[r].imag();
            }
        }
    }
    return NSSTAB_OK;
}

int nsstab_dense_schur_ordered(int n, const double* A, double thr, double* T, double* Z, int* p) {
    if (n < 1 || !A || !T || !Z || !p) return bad_arg("nsstab_dense_schur_ordered: bad argument");
    std::memcpy(T, A, (size_t)n * n * sizeof(double));
    std::memset(Z, 0, (size_t)n * n * sizeof(double));
    for (int i = 0; i < n; ++i) Z[i + (size_t)i * n] = 1.0;
    dense::hessenberg(n, T, Z);
    if (dense::schur(n, T, Z) != 0) {
        set_error("nsstab_dense_schur_ordered: QR iteration did not converge");
        return NSSTAB_ERR_NUMERICAL;
    }
    const int k = dense::schur_reorder(n, T, Z, [&](dense::cd e) { return std::abs(e) >= thr; });
    if (k < 0) {
        set_error("nsstab_dense_schur_ordered: ill-conditioned block swap");
        return NSSTAB_ERR_NUMERICAL;
    }
    *p = k;
    return NSSTAB_OK;
}

}  // extern "C"
