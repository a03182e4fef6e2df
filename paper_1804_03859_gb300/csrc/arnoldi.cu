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
#include <functional>
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
    const int nb = st->members();
    std::vector<long> nm(nb, n);
    auto prod = [&](const double* const* in, double* const* out) { return st->step_linear_ptrs(in, out, nsteps); };
    return arnoldi_members_run(prod, nb, nm.data(), stream, v0, m, nev, tol, max_restarts, outs);
}

int arnoldi_members_run(const std::function<int(const double* const*, double* const*)>& prod, int nb,
                        const long* nm, cudaStream_t stream, const double* const* v0, int m, int nev, double tol,
                        int max_restarts, std::vector<ArnoldiOut>& outs) {
    const double delta = 0.05;   // wanted set |mu| >= 1 - delta (Sec. 3.2.2)
    outs.resize(nb);
    const int ldb = m + 1;
    long nmax = 0;
    std::vector<size_t> off(nb + 1, 0);   // member b's basis at Vall + off[b]
    for (int b = 0; b < nb; ++b) {
        nmax = std::max(nmax, nm[b]);
        off[b + 1] = off[b] + (size_t)nm[b] * (m + 1);
    }
    DevBuf Vall, tmp, Cd;
    NS_CUDA(cudaMalloc(&Vall.p, off[nb] * sizeof(double)));
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
            mem[b].V = Vall.p + off[b];
            mem[b].B.assign((size_t)ldb * m, 0.0);
            NS_CUDA(cudaMemcpyAsync(mem[b].V, v0[b], nm[b] * sizeof(double), cudaMemcpyDeviceToDevice, stream));
            V0[b] = mem[b].V;
            W0[b] = mem[b].V;
        }
        NS_TRY(cgs2_batch(nb, V0.data(), nmax, nmax, j0.data(), W0.data(), h.data(), 0, beta.data(), gs, stream,
                          nm));
        for (int b = 0; b < nb; ++b) {
            if (!(beta[b] > 0.0) || !std::isfinite(beta[b])) {
                set_error("arnoldi_eigs: starting vector has zero or non-finite norm");
                return NSSTAB_ERR_INVALID_ARG;
            }
            inv[b] = 1.0 / beta[b];
        }
        NS_TRY(scale_batch(nb, W0.data(), nmax, inv.data(), gs, stream, nm));
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
            in[b] = M.V + (size_t)M.j * nm[b];
            out[b] = M.V + (size_t)(M.j + 1) * nm[b];
            wv[b] = out[b];
            Vp[b] = M.V;
            jv[b] = M.j + 1;
        }
        if (active == 0) break;
        // one batched product with M, one batched CGS2
        NS_TRY(prod(in.data(), out.data()));
        NS_TRY(cgs2_batch(nb, Vp.data(), nmax, nmax, jv.data(), wv.data(), H.data(), m + 1, beta.data(), gs, stream,
                          nm));
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
        NS_TRY(scale_batch(nb, scale_ptr.data(), nmax, inv.data(), gs, stream, nm));
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
            const long n = nm[b];
            if (!tmp.p) NS_CUDA(cudaMalloc(&tmp.p, (size_t)nmax * m * sizeof(double)));
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
            NS_TRY(basis_combine(M.V, nm[b], nm[b], mm, Cd.p, M.k, o.eigvecs, nm[b], stream));
            NS_CUDA(cudaStreamSynchronize(stream));
        }
    }
    NS_CUDA(cudaStreamSynchronize(stream));
    return NSSTAB_OK;
}

// Block Krylov-Schur with a block of b vectors per product with M, for
// every parameter set of the batched stepper at once (b = members / sets;
// the b members of a set share its base flow).  The b new columns of a
// round are orthogonalised against the basis by blocked CGS2 (two
// tall-skinny passes, each reading the basis once for all b columns) and
// then against each other, which gives column c the same coefficients as
// Gram-Schmidt against all columns before it, so M V_j = V_{j+b} B with B
// banded (b sub-diagonals); the residual of a Ritz pair (theta, V y) is
// ||R y||, R the b rows of B below the square part.
// The restart keeps the wanted Schur vectors and the b residual columns:
// M V_p = V_p T_p + V_res (R Z_p), the block form of Sec. 3.2.2's
// decomposition (Eqs. 60-63 have b = 1).  The sets' processes advance in
// lockstep rounds: one batched product with M over the b new columns of
// every unfinished set, one batched block Gram-Schmidt across the sets,
// then the b intra-block steps.  A finished set leaves the rounds.
namespace {
struct BlockProb {
    double* V = nullptr;            // device basis, n x (m + 2 b)
    std::vector<double> B;          // projected matrix, (m + 2 b) x (m + b) column-major
    int j = 0, mm = 0, k = 0, conv = 0, restarts = 0, matvec = 0;
    bool done = false, breakdown = false;
    std::vector<double> T, Z, res;
    std::vector<dense::cd> ev;
    std::vector<int> order;
};
}  // namespace

int block_arnoldi_run(StepperBase* st, cudaStream_t stream, long n, const double* const* v0, int m, int nev,
                      double tol, int max_restarts, int nsteps, std::vector<ArnoldiOut>& outs) {
    const double delta = 0.05;
    const int S = st->sets();
    const int b = st->members() / S;
    const int ncol = m + 2 * b;      // basis columns held
    const int ldb = m + 2 * b;       // rows of the projected matrix
    outs.resize(S);
    DevBuf Vd, tmp, Cd;
    NS_CUDA(cudaMalloc(&Vd.p, (size_t)S * n * ncol * sizeof(double)));
    NS_CUDA(cudaMalloc(&Cd.p, (size_t)ncol * ncol * sizeof(double)));
    NS_CUDA(cudaMalloc(&tmp.p, (size_t)n * ncol * sizeof(double)));
    GsBatch gs;
    struct Release {
        GsBatch& g;
        ~Release() { g.release(); }
    } rel{gs};
    NS_TRY(gs.alloc(S, ncol * b));   // the block passes' coefficients: (m + b) x b per set
    std::vector<BlockProb> pr(S);
    std::vector<const double*> Vp(S), Vb(S);
    std::vector<double*> wv(S), sp(S), wb(S);
    std::vector<int> jv(S), jb(S);
    const int ldhb = ncol * b;
    std::vector<double> H((size_t)S * ncol), HB((size_t)S * ldhb), beta(S), nrm(S), inv(S);
    for (int s = 0; s < S; ++s) {
        pr[s].V = Vd.p + (size_t)s * n * ncol;
        pr[s].B.assign((size_t)ldb * (m + b), 0.0);
        Vp[s] = pr[s].V;
    }
    // orthonormal start blocks: column i of every set in one batched CGS2
    for (int i = 0; i < b; ++i) {
        for (int s = 0; s < S; ++s) {
            wv[s] = pr[s].V + (size_t)i * n;
            NS_CUDA(cudaMemcpyAsync(wv[s], v0[(size_t)s * b + i], n * sizeof(double), cudaMemcpyDeviceToDevice,
                                    stream));
            jv[s] = 0;
        }
        NS_TRY(cgs2_batch(S, Vp.data(), n, n, jv.data(), wv.data(), H.data(), ncol, nrm.data(), gs, stream));
        std::fill(jv.begin(), jv.end(), i);
        NS_TRY(cgs2_batch(S, Vp.data(), n, n, jv.data(), wv.data(), H.data(), ncol, beta.data(), gs, stream));
        for (int s = 0; s < S; ++s) {
            if (!(nrm[s] > 0.0) || !std::isfinite(nrm[s]) || !(beta[s] > 1e-10 * nrm[s])) {
                set_error("block_arnoldi_eigs: start vectors are zero, non-finite or linearly dependent");
                return NSSTAB_ERR_INVALID_ARG;
            }
            inv[s] = 1.0 / beta[s];
        }
        NS_TRY(scale_batch(S, wv.data(), n, inv.data(), gs, stream));
    }
    std::vector<const double*> in((size_t)S * b);
    std::vector<double*> outp((size_t)S * b);
    while (true) {
        int active = 0;
        for (int s = 0; s < S; ++s) {
            BlockProb& P = pr[s];
            for (int i = 0; i < b; ++i) {
                in[(size_t)s * b + i] = P.done ? nullptr : P.V + (size_t)(P.j + i) * n;
                outp[(size_t)s * b + i] = P.done ? nullptr : P.V + (size_t)(P.j + b + i) * n;
            }
            if (!P.done) {
                ++active;
                P.matvec += b;
                P.breakdown = false;
            }
        }
        if (active == 0) break;
        NS_TRY(st->step_linear_ptrs(in.data(), outp.data(), nsteps));
        // block Gram-Schmidt: the b new columns of every set against its
        // J = j + b orthonormal columns in two tall-skinny passes (one read
        // of the basis per pass for all b columns) ...
        for (int s = 0; s < S; ++s) {
            const BlockProb& P = pr[s];
            jb[s] = P.done ? -1 : P.j + b;
            wb[s] = P.done ? nullptr : P.V + (size_t)(P.j + b) * n;
        }
        NS_TRY(bcgs2_batch(S, Vp.data(), n, n, jb.data(), wb.data(), n, b, HB.data(), ldhb, gs, stream));
        // ... then CGS2 of each new column against the block's earlier ones:
        // M v_{j+i} = V_J HB[:, i] + sum_{r < i} q_r h_r + beta q_i, the same
        // coefficients as column-by-column Gram-Schmidt against all J + i
        // columns (q_r is orthogonal to V_J)
        for (int i = 0; i < b; ++i) {
            for (int s = 0; s < S; ++s) {
                const BlockProb& P = pr[s];
                jv[s] = P.done ? -1 : i;
                Vb[s] = P.V + (size_t)(P.j + b) * n;
                wv[s] = P.done ? nullptr : P.V + (size_t)(P.j + b + i) * n;
            }
            NS_TRY(cgs2_batch(S, Vb.data(), n, n, jv.data(), wv.data(), H.data(), ncol, beta.data(), gs, stream));
            for (int s = 0; s < S; ++s) {
                BlockProb& P = pr[s];
                sp[s] = nullptr;
                inv[s] = 0.0;
                if (P.done) continue;
                const int J = P.j + b, c = J + i, col = P.j + i;
                double hn = 0.0;
                for (int r = 0; r < J; ++r) {
                    const double h = HB[(size_t)s * ldhb + (size_t)r * b + i];
                    P.B[r + (size_t)col * ldb] = h;
                    hn += h * h;
                }
                for (int r = 0; r < i; ++r) {
                    const double h = H[(size_t)s * ncol + r];
                    P.B[J + r + (size_t)col * ldb] = h;
                    hn += h * h;
                }
                P.B[c + (size_t)col * ldb] = beta[s];
                if (!std::isfinite(beta[s]) || !std::isfinite(hn)) {
                    set_error("block_arnoldi_eigs: non-finite values in the Krylov basis");
                    return NSSTAB_DIVERGED;
                }
                if (beta[s] <= 1e-14 * std::max(1.0, std::sqrt(hn))) {
                    P.breakdown = true;   // invariant subspace: the factorisation is exact
                    P.B[c + (size_t)col * ldb] = 0.0;
                } else {
                    sp[s] = wv[s];
                    inv[s] = 1.0 / beta[s];
                }
            }
            NS_TRY(scale_batch(S, sp.data(), n, inv.data(), gs, stream));
        }
        for (int s = 0; s < S; ++s) {
            BlockProb& P = pr[s];
            if (P.done) continue;
            P.j += b;
            if (P.j < m && !P.breakdown) continue;
            // full factorisation of order mm: Schur form, Ritz values, residuals ||R y||
            const int mm = P.j;
            P.mm = mm;
            P.T.assign((size_t)mm * mm, 0.0);
            P.Z.assign((size_t)mm * mm, 0.0);
            for (int c = 0; c < mm; ++c) {
                P.Z[c + (size_t)c * mm] = 1.0;
                for (int r = 0; r < mm; ++r) P.T[r + (size_t)c * mm] = P.B[r + (size_t)c * ldb];
            }
            dense::hessenberg(mm, P.T.data(), P.Z.data());
            if (dense::schur(mm, P.T.data(), P.Z.data()) != 0) {
                set_error("block_arnoldi_eigs: QR iteration on the projected matrix did not converge");
                return NSSTAB_ERR_NUMERICAL;
            }
            P.ev = dense::schur_eigenvalues(mm, P.T.data());
            P.order = leading_order(P.ev);
            P.k = take_leading(P.ev, P.order, nev);
            P.res.assign(P.k, 0.0);
            P.conv = 0;
            for (int s2 = 0; s2 < P.k; ++s2) {
                const std::vector<dense::cd> y = ritz_vector(mm, P.T.data(), P.Z.data(), P.ev, P.order[s2]);
                double r2 = 0.0;
                for (int q = 0; q < b; ++q) {
                    dense::cd acc = 0.0;
                    for (int c = 0; c < mm; ++c) acc += P.B[(mm + q) + (size_t)c * ldb] * y[c];
                    r2 += std::norm(acc);
                }
                P.res[s2] = std::sqrt(r2);
                if (P.res[s2] <= tol) ++P.conv;
            }
            if (P.conv >= P.k || P.restarts >= max_restarts || P.breakdown) {
                P.done = true;
                outs[s].done_at = steady_seconds();
                continue;
            }
            // restart: keep p Schur vectors and the b residual columns.  A
            // block basis of mm columns holds only mm / b powers of M, so
            // keeping just the values with |mu| >= 1 - delta (the
            // single-vector rule) can leave too small a space to converge a
            // clustered spectrum (seen to stall); keep at least half of the
            // basis beyond the k wanted.
            int p = 0;
            for (const auto& e : P.ev)
                if (std::abs(e) >= 1.0 - delta) ++p;
            p = std::max(P.k, std::min(std::max(p, P.k + (mm - P.k) / 2), mm - b));
            std::vector<double> mags(mm);
            for (int s2 = 0; s2 < mm; ++s2) mags[s2] = std::abs(P.ev[s2]);
            std::sort(mags.begin(), mags.end(), std::greater<double>());
            const double thr = mags[p - 1] * (1.0 - 1e-12);
            const int psel =
                dense::schur_reorder(mm, P.T.data(), P.Z.data(), [&](dense::cd e) { return std::abs(e) >= thr; });
            if (psel <= 0 || psel + b > mm) {
                set_error("block_arnoldi_eigs: Schur reordering failed");
                return NSSTAB_ERR_NUMERICAL;
            }
            p = psel;
            NS_CUDA(cudaMemcpyAsync(Cd.p, P.Z.data(), (size_t)mm * p * sizeof(double), cudaMemcpyHostToDevice,
                                    stream));
            NS_TRY(basis_combine(P.V, n, n, mm, Cd.p, p, tmp.p, n, stream));
            NS_CUDA(cudaMemcpyAsync(P.V, tmp.p, (size_t)n * p * sizeof(double), cudaMemcpyDeviceToDevice, stream));
            NS_CUDA(cudaMemcpyAsync(P.V + (size_t)p * n, P.V + (size_t)mm * n, (size_t)n * b * sizeof(double),
                                    cudaMemcpyDeviceToDevice, stream));
            std::vector<double> Bn((size_t)ldb * (m + b), 0.0);
            for (int c = 0; c < p; ++c) {
                for (int r = 0; r < p; ++r) Bn[r + (size_t)c * ldb] = P.T[r + (size_t)c * mm];
                for (int q = 0; q < b; ++q) {
                    double acc = 0.0;
                    for (int r = 0; r < mm; ++r) acc += P.B[(mm + q) + (size_t)r * ldb] * P.Z[r + (size_t)c * mm];
                    Bn[(p + q) + (size_t)c * ldb] = acc;
                }
            }
            P.B.swap(Bn);
            NS_CUDA(cudaStreamSynchronize(stream));   // Z upload done before Cd is reused
            P.j = p;
            ++P.restarts;
        }
    }
    for (int s = 0; s < S; ++s) {
        BlockProb& P = pr[s];
        ArnoldiOut& out = outs[s];
        out.n_eig = P.k;
        out.n_conv = P.conv;
        out.n_matvec = P.matvec;
        out.restarts = P.restarts;
        out.mu.resize(P.k);
        out.resid = P.res;
        for (int s2 = 0; s2 < P.k; ++s2) out.mu[s2] = P.ev[P.order[s2]];
        out.status = (P.conv >= P.k) ? NSSTAB_OK : NSSTAB_NOT_CONVERGED;
        if (out.eigvecs) {
            const int mm = P.mm;
            std::vector<double> Y((size_t)mm * P.k, 0.0);
            int s2 = 0;
            while (s2 < P.k) {
                const std::vector<dense::cd> y = ritz_vector(mm, P.T.data(), P.Z.data(), P.ev, P.order[s2]);
                if (P.ev[P.order[s2]].imag() != 0.0 && s2 + 1 < P.k) {
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
            NS_TRY(basis_combine(P.V, n, n, mm, Cd.p, P.k, out.eigvecs, n, stream));
            NS_CUDA(cudaStreamSynchronize(stream));
        }
    }
    NS_CUDA(cudaStreamSynchronize(stream));
    return NSSTAB_OK;
}

}  // namespace nsstab
