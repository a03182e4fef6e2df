// Arnoldi factorisation (Sec. 3.2.1, Algorithm 1, Eq. 57) with CGS2 and the
// Krylov-Schur restart (Sec. 3.2.2, Eqs. 60-63) around the matrix-free
// propagator M v = exp(T A) v of the stepper.
//
// Device / host split: every length-n vector (the basis V, the products
// M v, the Gram-Schmidt updates) stays on the GPU; only the j+1 projection
// coefficients and beta of each step come back (one small D2H copy per
// Krylov step), and the m x m projected matrix is factorised on the host in
// FP64 (dense_eig.cpp).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "arnoldi.h"
#include "dense_eig.h"

namespace nsstab {

namespace {

struct DevBuf {
    double* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

// leading order: |mu| descending, then Im(mu) descending
std::vector<int> leading_order(const std::vector<dense::cd>& ev) {
    std::vector<int> idx(ev.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        const double ma = std::abs(ev[a]), mb = std::abs(ev[b]);
        if (ma != mb) return ma > mb;
        return ev[a].imag() > ev[b].imag();
    });
    return idx;
}

// number of leading values to keep so that no conjugate pair is split
int take_leading(const std::vector<dense::cd>& ev, const std::vector<int>& order, int nev) {
    int k = std::min<int>(nev, (int)ev.size());
    if (k > 0 && k < (int)ev.size()) {
        const dense::cd last = ev[order[k - 1]];
        const dense::cd next = ev[order[k]];
        if (last.imag() > 0 && std::abs(next - std::conj(last)) <= 1e-12 * std::max(1.0, std::abs(last))) ++k;
    }
    return k;
}

// eigenvector (unit norm, length mm) of the Schur form for eigenvalue index i
std::vector<dense::cd> ritz_vector(int mm, const double* Tm, const double* Zm, const std::vector<dense::cd>& ev, int i) {
    // block start of eigenvalue i: a 2x2 block starts at i if T(i+1,i) != 0,
    // or at i-1 if T(i,i-1) != 0
    if (i > 0 && Tm[i + (size_t)(i - 1) * mm] != 0.0) {
        std::vector<dense::cd> y = dense::schur_eigenvector(mm, Tm, Zm, i - 1, ev[i - 1]);
        for (auto& v : y) v = std::conj(v);
        return y;
    }
    return dense::schur_eigenvector(mm, Tm, Zm, i, ev[i]);
}

}  // namespace

int arnoldi_run(StepperBase* st, GsWork& gs, cudaStream_t stream, const nsstab_config& cfg, long n,
                const double* v0, int m, int nev, double tol, int max_restarts, int nsteps, ArnoldiOut& out) {
    const double delta = 0.05;   // wanted set |mu| >= 1 - delta (Sec. 3.2.2)
    DevBuf V, tmp, Cd;
    NS_CUDA(cudaMalloc(&V.p, (size_t)n * (m + 1) * sizeof(double)));
    NS_CUDA(cudaMalloc(&Cd.p, (size_t)(m + 1) * (m + 1) * sizeof(double)));
    NS_TRY(gs.alloc(m + 1));
    double nrm = 0.0;
    NS_TRY(vec_norm(v0, n, &nrm, gs, stream));
    if (!(nrm > 0.0) || !std::isfinite(nrm)) {
        set_error("arnoldi_eigs: starting vector has zero or non-finite norm");
        return NSSTAB_ERR_INVALID_ARG;
    }
    NS_TRY(vec_scale(V.p, v0, n, 1.0 / nrm, stream));
    const int ldb = m + 1;
    std::vector<double> B((size_t)ldb * m, 0.0), h(m + 1);
    auto Bat = [&](int i, int j) -> double& { return B[i + (size_t)j * ldb]; };
    int j0 = 0, restarts = 0, matvec = 0;
    bool hessenberg_form = true;
    std::vector<double> Tm, Zm;
    std::vector<dense::cd> ev;
    std::vector<int> order;
    int k = 0, mm = m;
    double betam = 0.0;
    bool breakdown = false;
    std::vector<double> res;
    while (true) {
        mm = m;
        breakdown = false;
        for (int j = j0; j < m; ++j) {
            double* vj = V.p + (size_t)j * n;
            double* w = V.p + (size_t)(j + 1) * n;
            NS_TRY(st->step_linear(vj, w, nsteps));
            ++matvec;
            double beta = 0.0;
            NS_TRY(cgs2(V.p, n, n, j + 1, w, h.data(), &beta, gs, stream));
            double hn = 0.0;
            for (int i = 0; i <= j; ++i) {
                Bat(i, j) = h[i];
                hn += h[i] * h[i];
            }
            Bat(j + 1, j) = beta;
            if (!std::isfinite(beta)) {
                set_error("arnoldi_eigs: non-finite values in the Krylov basis");
                out.status = NSSTAB_DIVERGED;
                return NSSTAB_DIVERGED;
            }
            if (beta <= 1e-14 * std::max(1.0, std::sqrt(hn))) {   // invariant subspace
                mm = j + 1;
                breakdown = true;
                break;
            }
            NS_TRY(vec_scale(w, w, n, 1.0 / beta, stream));
        }
        betam = breakdown ? 0.0 : Bat(mm, mm - 1);
        // Schur form of the projected matrix B_mm
        Tm.assign((size_t)mm * mm, 0.0);
        Zm.assign((size_t)mm * mm, 0.0);
        for (int j = 0; j < mm; ++j) {
            Zm[j + (size_t)j * mm] = 1.0;
            for (int i = 0; i < mm; ++i) Tm[i + (size_t)j * mm] = Bat(i, j);
        }
        if (!hessenberg_form) dense::hessenberg(mm, Tm.data(), Zm.data());
        if (dense::schur(mm, Tm.data(), Zm.data()) != 0) {
            set_error("arnoldi_eigs: QR iteration on the projected matrix did not converge");
            return NSSTAB_ERR_NUMERICAL;
        }
        ev = dense::schur_eigenvalues(mm, Tm.data());
        order = leading_order(ev);
        k = take_leading(ev, order, nev);
        res.assign(k, 0.0);
        int conv = 0;
        for (int s = 0; s < k; ++s) {
            const std::vector<dense::cd> y = ritz_vector(mm, Tm.data(), Zm.data(), ev, order[s]);
            res[s] = std::abs(betam * y[mm - 1]);   // Eq. 63
            if (res[s] <= tol) ++conv;
        }
        out.n_conv = conv;
        if (conv >= k || restarts >= max_restarts || breakdown) break;
        // ---- Krylov-Schur restart: keep the p wanted Ritz values
        int p = 0;
        for (const auto& e : ev)
            if (std::abs(e) >= 1.0 - delta) ++p;
        p = std::max(k, std::min(p, mm / 2));
        {
            const dense::cd thr_mu = ev[order[p - 1]];
            if (thr_mu.imag() != 0.0 && p < mm) {
                for (int s = p; s < mm; ++s)
                    if (std::abs(ev[order[s]] - std::conj(thr_mu)) <= 1e-12 * std::max(1.0, std::abs(thr_mu))) {
                        ++p;
                        break;
                    }
            }
        }
        std::vector<double> mags(mm);
        for (int s = 0; s < mm; ++s) mags[s] = std::abs(ev[s]);
        std::sort(mags.begin(), mags.end(), std::greater<double>());
        const double thr = mags[p - 1] * (1.0 - 1e-12);
        const int psel = dense::schur_reorder(mm, Tm.data(), Zm.data(), [&](dense::cd e) { return std::abs(e) >= thr; });
        if (psel <= 0 || psel >= mm) {
            set_error("arnoldi_eigs: Schur reordering failed");
            return NSSTAB_ERR_NUMERICAL;
        }
        p = psel;
        // V_p <- V_mm Z(:, :p), v_{p+1} <- v_{mm+1}
        if (!tmp.p) NS_CUDA(cudaMalloc(&tmp.p, (size_t)n * m * sizeof(double)));
        NS_CUDA(cudaMemcpyAsync(Cd.p, Zm.data(), (size_t)mm * p * sizeof(double), cudaMemcpyHostToDevice, stream));
        NS_TRY(basis_combine(V.p, n, n, mm, Cd.p, p, tmp.p, n, stream));
        NS_CUDA(cudaMemcpyAsync(V.p, tmp.p, (size_t)n * p * sizeof(double), cudaMemcpyDeviceToDevice, stream));
        NS_CUDA(cudaMemcpyAsync(V.p + (size_t)p * n, V.p + (size_t)mm * n, (size_t)n * sizeof(double),
                                cudaMemcpyDeviceToDevice, stream));
        // B <- [[S11], [b^T Z(:, :p)]] with b = beta_m e_m
        std::fill(B.begin(), B.end(), 0.0);
        for (int j = 0; j < p; ++j) {
            for (int i = 0; i < p; ++i) Bat(i, j) = Tm[i + (size_t)j * mm];
            Bat(p, j) = betam * Zm[(mm - 1) + (size_t)j * mm];
        }
        NS_CUDA(cudaStreamSynchronize(stream));   // Zm upload done before reuse
        j0 = p;
        hessenberg_form = false;
        ++restarts;
    }
    // outputs in leading order
    out.n_eig = k;
    out.n_matvec = matvec;
    out.restarts = restarts;
    out.mu.resize(k);
    out.resid = res;
    for (int s = 0; s < k; ++s) out.mu[s] = ev[order[s]];
    if (out.eigvecs) {
        // columns of Y (mm x k): real vector, or Re / Im of a conjugate pair
        std::vector<double> Y((size_t)mm * k, 0.0);
        int s = 0;
        while (s < k) {
            const std::vector<dense::cd> y = ritz_vector(mm, Tm.data(), Zm.data(), ev, order[s]);
            if (ev[order[s]].imag() != 0.0 && s + 1 < k) {
                for (int i = 0; i < mm; ++i) {
                    Y[i + (size_t)s * mm] = y[i].real();
                    Y[i + (size_t)(s + 1) * mm] = y[i].imag();
                }
                s += 2;
            } else {
                for (int i = 0; i < mm; ++i) Y[i + (size_t)s * mm] = y[i].real();
                s += 1;
            }
        }
        NS_CUDA(cudaMemcpyAsync(Cd.p, Y.data(), Y.size() * sizeof(double), cudaMemcpyHostToDevice, stream));
        NS_TRY(basis_combine(V.p, n, n, mm, Cd.p, k, out.eigvecs, n, stream));
    }
    NS_CUDA(cudaStreamSynchronize(stream));
    out.status = (out.n_conv >= k) ? NSSTAB_OK : NSSTAB_NOT_CONVERGED;
    (void)cfg;
    return out.status;
}

}  // namespace nsstab
