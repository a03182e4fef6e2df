// Newton-Krylov fixed-point solver (Sec. 3.1.2, Eq. 43) around the stepper:
//   q <- q - (I - M)^{-1} (q - Phi_T(q)),
// Phi_T = T/dt nonlinear steps, M its Jacobian at q: by default the exact
// discrete tangent (a two-member stepper advancing the trajectory from q and
// the perturbation linearised about each of its points, co-integration), or
// the linearised propagator about q itself (frozen base flow: the exact
// Jacobian at a steady state, O(||q - Phi_T(q)||) away from it near one,
// one march per product instead of two).  The linear system is
// solved by restarted GMRES(m) whose Arnoldi basis is orthogonalised with
// CGS2 on the GPU; the (m+1) x m least-squares problem is reduced by Givens
// rotations on the host.  The products with M may come from a second
// stepper (for instance FP32) while the residual and the nonlinear map use
// the first (FP64): an inexact Newton method with an FP64 residual.
#include <cmath>
#include <functional>
#include <vector>

#include "newton.h"

namespace nsstab {

namespace {

struct DevBuf {
    double* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

using Product = std::function<int(const double*, double*)>;   // w = M v

// x = GMRES(m) solution of (I - M) x = b from x = 0.
int gmres_dev(const Product& Mv, long n, const double* b, double* x, int m, double rtol, int max_restarts,
              double* V, double* r, double* t, double* Cd, GsWork& gs, cudaStream_t stream, int* nmv) {
    double beta0 = 0.0;
    NS_TRY(vec_norm(b, n, &beta0, gs, stream));
    NS_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), stream));
    if (beta0 == 0.0) return NSSTAB_OK;
    NS_CUDA(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h(m + 1), y(m);
    for (int rs = 0; rs <= max_restarts; ++rs) {
        double beta = 0.0;
        NS_TRY(vec_norm(r, n, &beta, gs, stream));
        if (beta <= rtol * beta0) break;
        NS_TRY(vec_scale(V, r, n, 1.0 / beta, stream));
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        bool conv = false;
        for (int j = 0; j < m; ++j) {
            double* vj = V + (size_t)j * n;
            double* w = V + (size_t)(j + 1) * n;
            NS_TRY(Mv(vj, w));                                 // w = M v_j
            ++*nmv;
            NS_TRY(vec_axpby(w, 1.0, vj, -1.0, w, n, stream));  // w = (I - M) v_j
            double hn = 0.0;
            NS_TRY(cgs2(V, n, n, j + 1, w, h.data(), &hn, gs, stream));
            for (int i = 0; i < j; ++i) {
                const double tt = cs[i] * h[i] + sn[i] * h[i + 1];
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
                h[i] = tt;
            }
            const double d = std::hypot(h[j], hn);
            cs[j] = d == 0.0 ? 1.0 : h[j] / d;
            sn[j] = d == 0.0 ? 0.0 : hn / d;
            h[j] = d;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; ++i) H[i + (size_t)j * (m + 1)] = h[i];
            k = j + 1;
            if (!std::isfinite(g[j + 1])) {
                set_error("newton_krylov_fixedpoint: non-finite values in GMRES");
                return NSSTAB_DIVERGED;
            }
            if (std::fabs(g[j + 1]) <= rtol * beta0 || hn == 0.0) {
                conv = true;
                break;
            }
            NS_TRY(vec_scale(w, w, n, 1.0 / hn, stream));
        }
        // y = R^{-1} g, x += V_k y
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int c = i + 1; c < k; ++c) s -= H[i + (size_t)c * (m + 1)] * y[c];
            y[i] = s / H[i + (size_t)i * (m + 1)];
        }
        NS_CUDA(cudaMemcpyAsync(Cd, y.data(), k * sizeof(double), cudaMemcpyHostToDevice, stream));
        NS_TRY(basis_combine(V, n, n, k, Cd, 1, t, n, stream));
        NS_TRY(vec_axpby(x, 1.0, x, 1.0, t, n, stream));
        NS_CUDA(cudaStreamSynchronize(stream));   // y staged before it is reused
        if (conv || rs == max_restarts) break;
        // r = b - (I - M) x
        NS_TRY(Mv(x, t));
        ++*nmv;
        NS_TRY(vec_axpby(t, 1.0, x, -1.0, t, n, stream));
        NS_TRY(vec_axpby(r, 1.0, b, -1.0, t, n, stream));
    }
    return NSSTAB_OK;
}

}  // namespace

int newton_run(StepperBase* st, StepperBase* lin, StepperBase* tan, cudaStream_t stream, long n, double* q,
               int nsteps, int m, double gmres_rtol, int max_restarts, double tol, int max_newton, double* res_out,
               int* iters_out, int* mv_out) {
    DevBuf V, r, x, t, u, Cd;
    NS_CUDA(cudaMalloc(&V.p, (size_t)n * (m + 1) * sizeof(double)));
    NS_CUDA(cudaMalloc(&r.p, n * sizeof(double)));
    NS_CUDA(cudaMalloc(&x.p, n * sizeof(double)));
    NS_CUDA(cudaMalloc(&t.p, n * sizeof(double)));
    NS_CUDA(cudaMalloc(&u.p, n * sizeof(double)));
    NS_CUDA(cudaMalloc(&Cd.p, (size_t)(m + 1) * sizeof(double)));
    GsWork gs;
    struct Release {
        GsWork& g;
        ~Release() { g.release(); }
    } rel{gs};
    NS_TRY(gs.alloc(m + 2));
    int nmv = 0, k = 0;
    double res = INFINITY;
    int status = NSSTAB_NOT_CONVERGED;
    for (k = 0; k <= max_newton; ++k) {
        NS_TRY(st->residual(q, &res));
        if (!std::isfinite(res)) {
            status = NSSTAB_DIVERGED;
            break;
        }
        if (res <= tol) {
            status = NSSTAB_OK;
            break;
        }
        if (k == max_newton) break;
        // r = q - Phi_T(q)
        NS_CUDA(cudaMemcpyAsync(u.p, q, n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
        NS_TRY(st->step_nonlinear(u.p, nsteps));
        NS_TRY(vec_axpby(r.p, 1.0, q, -1.0, u.p, n, stream));
        Product Mv;
        if (tan) {
            Mv = [&](const double* v, double* w) { return tan->tangent(q, v, w, nsteps); };
        } else {
            NS_TRY(lin->set_base(q));
            Mv = [&](const double* v, double* w) { return lin->step_linear(v, w, nsteps); };
        }
        NS_TRY(gmres_dev(Mv, n, r.p, x.p, m, gmres_rtol, max_restarts, V.p, u.p, t.p, Cd.p, gs, stream, &nmv));
        NS_TRY(vec_axpby(q, 1.0, q, -1.0, x.p, n, stream));
    }
    NS_CUDA(cudaStreamSynchronize(stream));
    *res_out = res;
    *iters_out = std::min(k, max_newton);
    *mv_out = nmv;
    return status;
}

}  // namespace nsstab
