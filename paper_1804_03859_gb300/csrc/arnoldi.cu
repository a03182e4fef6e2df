// Arnoldi factorisation (Sec. 3.2.1, Algorithm 1, Eq. 57) with CGS2 and the
// Krylov-Schur restart (Sec. 3.2.2, Eqs. 60-63) around the matrix-free
// propagator M v = exp(T A) v of the stepper.
//
// The driver runs the independent eigenproblems of every member of a batched
// stepper in lockstep rounds: each round is one batched product with M (one
// set of step kernels for all members still working), one batched CGS2 and,
// per member, the update of its projected matrix; a member whose
// factorisation is full is checked for convergence and either finishes or is
// restarted, and finished members leave the batch (their blocks return at
// once).  A single stepper is the batch of one.
//
// Device / host split: every length-n vector (the bases, the products, the
// Gram-Schmidt updates) stays on the GPU; per round only the coefficients
// and beta of each member come back (one small D2H copy), and the m x m
// projected matrices are factorised on the host in FP64 (dense_eig.cpp).
#include <algorithm>
#include <chrono>
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
    if (i > 0 && Tm[i + (size_t)(i - 1) * mm] != 0.0) {
        std::vector<dense::cd> y = dense::schur_eigenvector(mm, Tm, Zm, i - 1, ev[i - 1]);
        for (auto& v : y) v = std::conj(v);
        return y;
    }
    return dense::schur_eigenvector(mm, Tm, Zm, i, ev[i]);
}

// Per-member state of the Krylov process.
struct Member {
    double* V = nullptr;            // device basis, n x (m+1)
    std::vector<double> B;          // projected matrix, (m+1) x m column-major
    int j = 0;                      // columns filled
    int restarts = 0, matvec = 0;
    bool hessenberg = true;         // B is upper Hessenberg (no restart yet)
    bool done = false, breakdown = false;
    int mm = 0;                     // order of the last factorisation
    double betam = 0.0;
    std::vector<double> Tm, Zm;     // Schur form of B_mm
    std::vector<dense::cd> ev;
    std::vector<int> order;
    std::vector<double> res;
    int k = 0, conv = 0;
};

}  // namespace

double steady_seconds() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int arnoldi_batch_run(StepperBase* st, cudaStream_t stream, long n, const double* const* v0, int m, int nev,
                      double tol, int max_restarts, int nsteps, std::vector<ArnoldiOut>& outs) {
    const double delta = 0.05;   // wanted set |mu| >= 1 - delta (Sec. 3.2.2)
    const int nb = st->members();
    outs.resize(nb);
    const int ldb = m + 1;
    DevBuf Vall, tmp, Cd;
    NS_CUDA(cudaMalloc(&Vall.p, (size_t)nb * n * (m + 1) * sizeof(double)));
    NS_CUDA(cudaMalloc(&Cd.p, (size_t)(m + 1) * (m + 1) * sizeof(double)));
    GsBatch gs;
    struct Release {
        GsBatch& g;
        ~Release() { g.release(); }
    } rel{gs};
    NS_TRY(gs.alloc(nb, m + 1));
    std::vector<Member> mem(nb);
    // v_1 = v0 / ||v0|| for every member
    {
        std::vector<const double*> V0(nb);
        std::vector<double*> W0(nb);
        std::vector<int> j0(nb, 0);
        std::vector<double> h(1), beta(nb), inv(nb);
        for (int b = 0; b < nb; ++b) {
            mem[b].V = Vall.p + (size_t)b * n * (m + 1);
            mem[b].B.assign((size_t)ldb * m, 0.0);
            NS_CUDA(cudaMemcpyAsync(mem[b].V, v0[b], n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
            V0[b] = mem[b].V;
            W0[b] = mem[b].V;
        }
        NS_TRY(cgs2_batch(nb, V0.data(), n, n, j0.data(), W0.data(), h.data(), 0, beta.data(), gs, stream));
        for (int b = 0; b < nb; ++b) {
            if (!(beta[b] > 0.0) || !std::isfinite(beta[b])) {
                set_error("arnoldi_eigs: starting vector has zero or non-finite norm");
                return NSSTAB_ERR_INVALID_ARG;
            }
            inv[b] = 1.0 / beta[b];
        }
        NS_TRY(scale_batch(nb, W0.data(), n, inv.data(), gs, stream));
    }
    std::vector<const double*> in(nb);
    std::vector<double*> out(nb), wv(nb);
    std::vector<const double*> Vp(nb);
    std::vector<int> jv(nb);
    std::vector<double> H((size_t)nb * (m + 1)), beta(nb), inv(nb);
    while (true) {
        int active = 0;
        for (int b = 0; b < nb; ++b) {
            Member& M = mem[b];
            if (M.done) {
                in[b] = nullptr;
                out[b] = nullptr;
                jv[b] = -1;
                wv[b] = nullptr;
                Vp[b] = M.V;
                continue;
            }
            ++active;
            in[b] = M.V + (size_t)M.j * n;
            out[b] = M.V + (size_t)(M.j + 1) * n;
            wv[b] = out[b];
            Vp[b] = M.V;
            jv[b] = M.j + 1;
        }
        if (active == 0) break;
        // one batched product with M, one batched CGS2
        NS_TRY(st->step_linear_ptrs(in.data(), out.data(), nsteps));
        NS_TRY(cgs2_batch(nb, Vp.data(), n, n, jv.data(), wv.data(), H.data(), m + 1, beta.data(), gs, stream));
        std::fill(inv.begin(), inv.end(), 0.0);
        std::vector<double*> scale_ptr(nb, nullptr);
        for (int b = 0; b < nb; ++b) {
            Member& M = mem[b];
            if (M.done) continue;
            const int j = M.j;
            ++M.matvec;
            double hn = 0.0;
            for (int i = 0; i <= j; ++i) {
                M.B[i + (size_t)j * ldb] = H[(size_t)b * (m + 1) + i];
                hn += H[(size_t)b * (m + 1) + i] * H[(size_t)b * (m + 1) + i];
            }
            M.B[(j + 1) + (size_t)j * ldb] = beta[b];
            if (!std::isfinite(beta[b])) {
                set_error("arnoldi_eigs: non-finite values in the Krylov basis");
                return NSSTAB_DIVERGED;
            }
            M.j = j + 1;
            if (beta[b] <= 1e-14 * std::max(1.0, std::sqrt(hn))) {   // invariant subspace
                M.breakdown = true;
            } else {
                inv[b] = 1.0 / beta[b];
                scale_ptr[b] = out[b];
            }
        }
        NS_TRY(scale_batch(nb, scale_ptr.data(), n, inv.data(), gs, stream));
        // members with a full factorisation: Ritz pairs, convergence, restart
        for (int b = 0; b < nb; ++b) {
            Member& M = mem[b];
            if (M.done || (M.j < m && !M.breakdown)) continue;
            const int mm = M.j;
            M.mm = mm;
            M.betam = M.breakdown ? 0.0 : M.B[mm + (size_t)(mm - 1) * ldb];
            M.Tm.assign((size_t)mm * mm, 0.0);
            M.Zm.assign((size_t)mm * mm, 0.0);
            for (int jj = 0; jj < mm; ++jj) {
                M.Zm[jj + (size_t)jj * mm] = 1.0;
                for (int i = 0; i < mm; ++i) M.Tm[i + (size_t)jj * mm] = M.B[i + (size_t)jj * ldb];
            }
            if (!M.hessenberg) dense::hessenberg(mm, M.Tm.data(), M.Zm.data());
            if (dense::schur(mm, M.Tm.data(), M.Zm.data()) != 0) {
                set_error("arnoldi_eigs: QR iteration on the projected matrix did not converge");
                return NSSTAB_ERR_NUMERICAL;
            }
            M.ev = dense::schur_eigenvalues(mm, M.Tm.data());
            M.order = leading_order(M.ev);
            M.k = take_leading(M.ev, M.order, nev);
            M.res.assign(M.k, 0.0);
            M.conv = 0;
            for (int s = 0; s < M.k; ++s) {
                const std::vector<dense::cd> y = ritz_vector(mm, M.Tm.data(), M.Zm.data(), M.ev, M.order[s]);
                M.res[s] = std::abs(M.betam * y[mm - 1]);   // Eq. 63
                if (M.res[s] <= tol) ++M.conv;
            }
            if (M.conv >= M.k || M.restarts >= max_restarts || M.breakdown) {
                M.done = true;
                outs[b].done_at = steady_seconds();
                continue;
            }
            // ---- Krylov-Schur restart: keep the p wanted Ritz values
            int p = 0;
            for (const auto& e : M.ev)
                if (std::abs(e) >= 1.0 - delta) ++p;
            p = std::max(M.k, std::min(p, mm / 2));
            {
                const dense::cd thr_mu = M.ev[M.order[p - 1]];
                if (thr_mu.imag() != 0.0 && p < mm) {
                    for (int s = p; s < mm; ++s)
                        if (std::abs(M.ev[M.order[s]] - std::conj(thr_mu)) <= 1e-12 * std::max(1.0, std::abs(thr_mu))) {
                            ++p;
                            break;
                        }
                }
            }
            std::vector<double> mags(mm);
            for (int s = 0; s < mm; ++s) mags[s] = std::abs(M.ev[s]);
            std::sort(mags.begin(), mags.end(), std::greater<double>());
            const double thr = mags[p - 1] * (1.0 - 1e-12);
            const int psel =
                dense::schur_reorder(mm, M.Tm.data(), M.Zm.data(), [&](dense::cd e) { return std::abs(e) >= thr; });
            if (psel <= 0 || psel >= mm) {
                set_error("arnoldi_eigs: Schur reordering failed");
                return NSSTAB_ERR_NUMERICAL;
            }
            p = psel;
            // V_p <- V_mm Z(:, :p), v_{p+1} <- v_{mm+1}
            if (!tmp.p) NS_CUDA(cudaMalloc(&tmp.p, (size_t)n * m * sizeof(double)));
            NS_CUDA(cudaMemcpyAsync(Cd.p, M.Zm.data(), (size_t)mm * p * sizeof(double), cudaMemcpyHostToDevice,
                                    stream));
            NS_TRY(basis_combine(M.V, n, n, mm, Cd.p, p, tmp.p, n, stream));
            NS_CUDA(cudaMemcpyAsync(M.V, tmp.p, (size_t)n * p * sizeof(double), cudaMemcpyDeviceToDevice, stream));
            NS_CUDA(cudaMemcpyAsync(M.V + (size_t)p * n, M.V + (size_t)mm * n, (size_t)n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, stream));
            // B <- [[S11], [b^T Z(:, :p)]] with b = beta_m e_m
            std::fill(M.B.begin(), M.B.end(), 0.0);
            for (int jj = 0; jj < p; ++jj) {
                for (int i = 0; i < p; ++i) M.B[i + (size_t)jj * ldb] = M.Tm[i + (size_t)jj * mm];
                M.B[p + (size_t)jj * ldb] = M.betam * M.Zm[(mm - 1) + (size_t)jj * mm];
            }
            NS_CUDA(cudaStreamSynchronize(stream));   // Zm upload done before Cd is reused
            M.j = p;
            M.hessenberg = false;
            ++M.restarts;
        }
    }
    // outputs in leading order
    for (int b = 0; b < nb; ++b) {
        Member& M = mem[b];
        ArnoldiOut& o = outs[b];
        o.n_eig = M.k;
        o.n_conv = M.conv;
        o.n_matvec = M.matvec;
        o.restarts = M.restarts;
        o.mu.resize(M.k);
        o.resid = M.res;
        for (int s = 0; s < M.k; ++s) o.mu[s] = M.ev[M.order[s]];
        o.status = (o.n_conv >= o.n_eig) ? NSSTAB_OK : NSSTAB_NOT_CONVERGED;
        if (o.eigvecs) {
            const int mm = M.mm;
            // columns of Y (mm x k): real vector, or Re / Im of a conjugate pair
            std::vector<double> Y((size_t)mm * M.k, 0.0);
            int s = 0;
            while (s < M.k) {
                const std::vector<dense::cd> y = ritz_vector(mm, M.Tm.data(), M.Zm.data(), M.ev, M.order[s]);
                if (M.ev[M.order[s]].imag() != 0.0 && s + 1 < M.k) {
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
            NS_TRY(basis_combine(M.V, n, n, mm, Cd.p, M.k, o.eigvecs, n, stream));
            NS_CUDA(cudaStreamSynchronize(stream));
        }
    }
    NS_CUDA(cudaStreamSynchronize(stream));
    return NSSTAB_OK;
}

// Block Krylov-Schur for ONE eigenproblem with a block of b = members
// vectors per product with M (the batched stepper's members share one base
// flow).  Column c of the basis is orthogonalised by CGS2 against all
// columns before it, so M V_j = V_{j+b} B with B banded (b sub-diagonals);
// the residual of a Ritz pair (theta, V y) is ||R y||, R the b rows of B
// below the square part.  The restart keeps the wanted Schur vectors and
// the b residual columns: M V_p = V_p T_p + V_res (R Z_p), the block form
// of Sec. 3.2.2's decomposition (Eqs. 60-63 have b = 1).
int block_arnoldi_run(StepperBase* st, cudaStream_t stream, long n, const double* const* v0, int m, int nev,
                      double tol, int max_restarts, int nsteps, ArnoldiOut& out) {
    const double delta = 0.05;
    const int b = st->members();
    const int ncol = m + 2 * b;      // basis columns held
    const int ldb = m + 2 * b;       // rows of the projected matrix
    DevBuf Vd, tmp, Cd;
    NS_CUDA(cudaMalloc(&Vd.p, (size_t)n * ncol * sizeof(double)));
    NS_CUDA(cudaMalloc(&Cd.p, (size_t)ncol * ncol * sizeof(double)));
    NS_CUDA(cudaMalloc(&tmp.p, (size_t)n * ncol * sizeof(double)));
    double* V = Vd.p;
    GsWork gs;
    struct Release {
        GsWork& g;
        ~Release() { g.release(); }
    } rel{gs};
    std::vector<double> h(ncol), B((size_t)ldb * (m + b), 0.0);
    // orthonormal start block
    for (int i = 0; i < b; ++i) {
        double* w = V + (size_t)i * n;
        NS_CUDA(cudaMemcpyAsync(w, v0[i], n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
        double nrm = 0.0, beta = 0.0;
        NS_TRY(vec_norm(w, n, &nrm, gs, stream));
        NS_TRY(cgs2(V, n, n, i, w, h.data(), &beta, gs, stream));
        if (!(nrm > 0.0) || !std::isfinite(nrm) || !(beta > 1e-10 * nrm)) {
            set_error("block_arnoldi_eigs: start vectors are zero, non-finite or linearly dependent");
            return NSSTAB_ERR_INVALID_ARG;
        }
        NS_TRY(vec_scale(w, w, n, 1.0 / beta, stream));
    }
    std::vector<const double*> in(b);
    std::vector<double*> outp(b);
    std::vector<double> T, Z;
    std::vector<dense::cd> ev;
    std::vector<int> order;
    std::vector<double> res;
    int j = 0, mm = 0, k = 0, conv = 0, restarts = 0, matvec = 0;
    while (true) {
        for (int i = 0; i < b; ++i) {
            in[i] = V + (size_t)(j + i) * n;
            outp[i] = V + (size_t)(j + b + i) * n;
        }
        NS_TRY(st->step_linear_ptrs(in.data(), outp.data(), nsteps));
        matvec += b;
        bool breakdown = false;
        for (int i = 0; i < b; ++i) {
            const int c = j + b + i, col = j + i;
            double beta = 0.0;
            NS_TRY(cgs2(V, n, n, c, V + (size_t)c * n, h.data(), &beta, gs, stream));
            double hn = 0.0;
            for (int r = 0; r < c; ++r) {
                B[r + (size_t)col * ldb] = h[r];
                hn += h[r] * h[r];
            }
            B[c + (size_t)col * ldb] = beta;
            if (!std::isfinite(beta)) {
                set_error("block_arnoldi_eigs: non-finite values in the Krylov basis");
                return NSSTAB_DIVERGED;
            }
            if (beta <= 1e-14 * std::max(1.0, std::sqrt(hn))) {
                breakdown = true;   // invariant subspace: the factorisation is exact
                B[c + (size_t)col * ldb] = 0.0;
            } else {
                NS_TRY(vec_scale(V + (size_t)c * n, V + (size_t)c * n, n, 1.0 / beta, stream));
            }
        }
        j += b;
        if (j < m && !breakdown) continue;
        // full factorisation of order mm: Schur form, Ritz values, residuals ||R y||
        mm = j;
        T.assign((size_t)mm * mm, 0.0);
        Z.assign((size_t)mm * mm, 0.0);
        for (int c = 0; c < mm; ++c) {
            Z[c + (size_t)c * mm] = 1.0;
            for (int r = 0; r < mm; ++r) T[r + (size_t)c * mm] = B[r + (size_t)c * ldb];
        }
        dense::hessenberg(mm, T.data(), Z.data());
        if (dense::schur(mm, T.data(), Z.data()) != 0) {
            set_error("block_arnoldi_eigs: QR iteration on the projected matrix did not converge");
            return NSSTAB_ERR_NUMERICAL;
        }
        ev = dense::schur_eigenvalues(mm, T.data());
        order = leading_order(ev);
        k = take_leading(ev, order, nev);
        res.assign(k, 0.0);
        conv = 0;
        for (int s2 = 0; s2 < k; ++s2) {
            const std::vector<dense::cd> y = ritz_vector(mm, T.data(), Z.data(), ev, order[s2]);
            double r2 = 0.0;
            for (int q = 0; q < b; ++q) {
                dense::cd acc = 0.0;
                for (int c = 0; c < mm; ++c) acc += B[(mm + q) + (size_t)c * ldb] * y[c];
                r2 += std::norm(acc);
            }
            res[s2] = std::sqrt(r2);
            if (res[s2] <= tol) ++conv;
        }
        if (conv >= k || restarts >= max_restarts || breakdown) break;
        // restart: keep p Schur vectors and the b residual columns.  A block
        // basis of mm columns holds only mm / b powers of M, so keeping just
        // the values with |mu| >= 1 - delta (the single-vector rule) can
        // leave too small a space to converge a clustered spectrum (seen to
        // stall); keep at least half of the basis beyond the k wanted.
        int p = 0;
        for (const auto& e : ev)
            if (std::abs(e) >= 1.0 - delta) ++p;
        p = std::max(k, std::min(std::max(p, k + (mm - k) / 2), mm - b));
        std::vector<double> mags(mm);
        for (int s2 = 0; s2 < mm; ++s2) mags[s2] = std::abs(ev[s2]);
        std::sort(mags.begin(), mags.end(), std::greater<double>());
        const double thr = mags[p - 1] * (1.0 - 1e-12);
        const int psel =
            dense::schur_reorder(mm, T.data(), Z.data(), [&](dense::cd e) { return std::abs(e) >= thr; });
        if (psel <= 0 || psel + b > mm) {
            set_error("block_arnoldi_eigs: Schur reordering failed");
            return NSSTAB_ERR_NUMERICAL;
        }
        p = psel;
        NS_CUDA(cudaMemcpyAsync(Cd.p, Z.data(), (size_t)mm * p * sizeof(double), cudaMemcpyHostToDevice, stream));
        NS_TRY(basis_combine(V, n, n, mm, Cd.p, p, tmp.p, n, stream));
        NS_CUDA(cudaMemcpyAsync(V, tmp.p, (size_t)n * p * sizeof(double), cudaMemcpyDeviceToDevice, stream));
        NS_CUDA(cudaMemcpyAsync(V + (size_t)p * n, V + (size_t)mm * n, (size_t)n * b * sizeof(double),
                                cudaMemcpyDeviceToDevice, stream));
        std::vector<double> Bn((size_t)ldb * (m + b), 0.0);
        for (int c = 0; c < p; ++c) {
            for (int r = 0; r < p; ++r) Bn[r + (size_t)c * ldb] = T[r + (size_t)c * mm];
            for (int q = 0; q < b; ++q) {
                double acc = 0.0;
                for (int r = 0; r < mm; ++r) acc += B[(mm + q) + (size_t)r * ldb] * Z[r + (size_t)c * mm];
                Bn[(p + q) + (size_t)c * ldb] = acc;
            }
        }
        B.swap(Bn);
        NS_CUDA(cudaStreamSynchronize(stream));   // Z upload done before Cd is reused
        j = p;
        ++restarts;
    }
    out.n_eig = k;
    out.n_conv = conv;
    out.n_matvec = matvec;
    out.restarts = restarts;
    out.mu.resize(k);
    out.resid = res;
    for (int s2 = 0; s2 < k; ++s2) out.mu[s2] = ev[order[s2]];
    out.status = (conv >= k) ? NSSTAB_OK : NSSTAB_NOT_CONVERGED;
    out.done_at = steady_seconds();
    if (out.eigvecs) {
        std::vector<double> Y((size_t)mm * k, 0.0);
        int s2 = 0;
        while (s2 < k) {
            const std::vector<dense::cd> y = ritz_vector(mm, T.data(), Z.data(), ev, order[s2]);
            if (ev[order[s2]].imag() != 0.0 && s2 + 1 < k) {
                for (int r = 0; r < mm; ++r) {
                    Y[r + (size_t)s2 * mm] = y[r].real();
                    Y[r + (size_t)(s2 + 1) * mm] = y[r].imag();
                }
                s2 += 2;
            } else {
                for (int r = 0; r < mm; ++r) Y[r + (size_t)s2 * mm] = y[r].real();
                s2 += 1;
            }
        }
        NS_CUDA(cudaMemcpyAsync(Cd.p, Y.data(), Y.size() * sizeof(double), cudaMemcpyHostToDevice, stream));
        NS_TRY(basis_combine(V, n, n, mm, Cd.p, k, out.eigvecs, n, stream));
    }
    NS_CUDA(cudaStreamSynchronize(stream));
    return NSSTAB_OK;
}

}  // namespace nsstab
