// Host FP64 dense eigen-solver: Householder Hessenberg reduction, Francis
// double-shift QR to real Schur form, eigenvectors by back substitution on
// the quasi-triangular factor, and reordering of the Schur form by direct
// swaps of adjacent diagonal blocks (Sylvester equation + QR).  The matrices
// are at most a few hundred wide (the Krylov dimension), so plain loops are
// adequate; no LAPACK is used.
#include "dense_eig.h"

#include <algorithm>
#include <cmath>
#include <limits>

namespace nsstab {
namespace dense {

namespace {

const double kEps = std::numeric_limits<double>::epsilon();

inline double& at(double* a, int n, int i, int j) { return a[i + (size_t)j * n]; }
inline double at(const double* a, int n, int i, int j) { return a[i + (size_t)j * n]; }

// Householder vector v (v[0] = 1 implied by storage of all L entries) and
// beta such that (I - beta v v^T) x = alpha e_1.
void house(const double* x, int L, double* v, double* beta) {
    double s = 0.0;
    for (int i = 0; i < L; ++i) s += x[i] * x[i];
    const double nrm = std::sqrt(s);
    for (int i = 0; i < L; ++i) v[i] = x[i];
    if (nrm == 0.0) {
        *beta = 0.0;
        return;
    }
    const double alpha = x[0] >= 0 ? -nrm : nrm;
    v[0] = x[0] - alpha;
    double vv = 0.0;
    for (int i = 0; i < L; ++i) vv += v[i] * v[i];
    *beta = vv > 0 ? 2.0 / vv : 0.0;
}

// rows r0..r0+L-1, columns c0..c1 of A: A <- (I - beta v v^T) A
void apply_left(int n, double* A, int r0, int L, int c0, int c1, const double* v, double beta) {
    if (beta == 0.0) return;
    for (int j = c0; j <= c1; ++j) {
        double s = 0.0;
        for (int i = 0; i < L; ++i) s += v[i] * at(A, n, r0 + i, j);
        s *= beta;
        for (int i = 0; i < L; ++i) at(A, n, r0 + i, j) -= s * v[i];
    }
}

// rows r0..r1, columns c0..c0+L-1 of A: A <- A (I - beta v v^T)
void apply_right(int n, double* A, int r0, int r1, int c0, int L, const double* v, double beta) {
    if (beta == 0.0) return;
    for (int i = r0; i <= r1; ++i) {
        double s = 0.0;
        for (int j = 0; j < L; ++j) s += at(A, n, i, c0 + j) * v[j];
        s *= beta;
        for (int j = 0; j < L; ++j) at(A, n, i, c0 + j) -= s * v[j];
    }
}

double norm1_est(int n, const double* A) {
    double m = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += std::fabs(at(A, n, i, j));
        m = std::max(m, s);
    }
    return m;
}

// Rotate the 2x2 diagonal block at (k, k) to upper-triangular form when its
// eigenvalues are real; leaves complex-pair blocks alone.
void standardize_2x2(int n, double* A, double* Z, int k) {
    const double a = at(A, n, k, k), b = at(A, n, k, k + 1);
    const double c = at(A, n, k + 1, k), d = at(A, n, k + 1, k + 1);
    if (c == 0.0) return;
    const double p = 0.5 * (a - d);
    const double disc = p * p + b * c;
    if (disc < 0.0) return;
    // real eigenvalue lam1 = (a+d)/2 + sign(p) sqrt(disc) (the larger-|.| root
    // relative to the mean avoids cancellation); eigenvector (lam1 - d, c)
    const double sq = std::sqrt(disc);
    const double lam = 0.5 * (a + d) + (p >= 0 ? sq : -sq);
    double x0 = lam - d, x1 = c;
    if (std::fabs(x0) + std::fabs(x1) == 0.0) {
        x0 = b;
        x1 = lam - a;
    }
    const double r = std::hypot(x0, x1);
    const double cs = x0 / r, sn = x1 / r;
    // G = [[cs, -sn], [sn, cs]], first column = eigenvector; A <- G^T A G
    for (int j = 0; j < n; ++j) {
        const double u = at(A, n, k, j), w = at(A, n, k + 1, j);
        at(A, n, k, j) = cs * u + sn * w;
        at(A, n, k + 1, j) = -sn * u + cs * w;
    }
    for (int i = 0; i < n; ++i) {
        const double u = at(A, n, i, k), w = at(A, n, i, k + 1);
        at(A, n, i, k) = cs * u + sn * w;
        at(A, n, i, k + 1) = -sn * u + cs * w;
    }
    for (int i = 0; i < n; ++i) {
        const double u = at(Z, n, i, k), w = at(Z, n, i, k + 1);
        at(Z, n, i, k) = cs * u + sn * w;
        at(Z, n, i, k + 1) = -sn * u + cs * w;
    }
    at(A, n, k + 1, k) = 0.0;
}

}  // namespace

void hessenberg(int n, double* A, double* Q) {
    std::vector<double> x(n), v(n);
    for (int k = 0; k + 2 < n; ++k) {
        const int L = n - k - 1;
        for (int i = 0; i < L; ++i) x[i] = at(A, n, k + 1 + i, k);
        double beta;
        house(x.data(), L, v.data(), &beta);
        if (beta == 0.0) continue;
        apply_left(n, A, k + 1, L, k, n - 1, v.data(), beta);
        apply_right(n, A, 0, n - 1, k + 1, L, v.data(), beta);
        apply_right(n, Q, 0, n - 1, k + 1, L, v.data(), beta);
        for (int i = k + 2; i < n; ++i) at(A, n, i, k) = 0.0;
    }
}

int schur(int n, double* A, double* Z) {
    const double anorm = std::max(norm1_est(n, A), std::numeric_limits<double>::min());
    int hi = n - 1;
    int iter = 0, total = 0;
    const int max_total = 100 * std::max(n, 10);
    double v[3];
    while (hi >= 0) {
        // find the start l of the active unreduced block ending at hi
        int l = hi;
        while (l > 0) {
            double s = std::fabs(at(A, n, l - 1, l - 1)) + std::fabs(at(A, n, l, l));
            if (s == 0.0) s = anorm;
            if (std::fabs(at(A, n, l, l - 1)) <= kEps * s) {
                at(A, n, l, l - 1) = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {            // 1x1 block converged
            --hi;
            iter = 0;
            continue;
        }
        if (l == hi - 1) {        // 2x2 block converged
            standardize_2x2(n, A, Z, hi - 1);
            hi -= 2;
            iter = 0;
            continue;
        }
        if (++total > max_total) return -1;
        ++iter;
        // double shift from the trailing 2x2 (exceptional shifts every 10 stalls)
        double s, t;
        if (iter % 10 == 0) {
            const double w = std::fabs(at(A, n, hi, hi - 1)) + std::fabs(at(A, n, hi - 1, hi - 2));
            s = 1.5 * w + at(A, n, hi, hi);
            t = w * w;
        } else {
            s = at(A, n, hi - 1, hi - 1) + at(A, n, hi, hi);
            t = at(A, n, hi - 1, hi - 1) * at(A, n, hi, hi) - at(A, n, hi - 1, hi) * at(A, n, hi, hi - 1);
        }
        // first column of (A - s1 I)(A - s2 I) restricted to the window
        double x = at(A, n, l, l) * at(A, n, l, l) + at(A, n, l, l + 1) * at(A, n, l + 1, l) - s * at(A, n, l, l) + t;
        double y = at(A, n, l + 1, l) * (at(A, n, l, l) + at(A, n, l + 1, l + 1) - s);
        double z = at(A, n, l + 1, l) * at(A, n, l + 2, l + 1);
        for (int k = l; k <= hi - 2; ++k) {
            const double xv[3] = {x, y, z};
            double beta;
            house(xv, 3, v, &beta);
            const int c0 = std::max(l, k - 1);
            apply_left(n, A, k, 3, c0, n - 1, v, beta);
            const int r1 = std::min(k + 3, hi);
            apply_right(n, A, 0, r1, k, 3, v, beta);
            apply_right(n, Z, 0, n - 1, k, 3, v, beta);
            if (k > l) {
                at(A, n, k + 1, k - 1) = 0.0;
                at(A, n, k + 2, k - 1) = 0.0;
            }
            x = at(A, n, k + 1, k);
            y = at(A, n, k + 2, k);
            if (k < hi - 2) z = at(A, n, k + 3, k);
        }
        {
            const double xv[2] = {x, y};
            double beta;
            house(xv, 2, v, &beta);
            apply_left(n, A, hi - 1, 2, hi - 2, n - 1, v, beta);
            apply_right(n, A, 0, hi, hi - 1, 2, v, beta);
            apply_right(n, Z, 0, n - 1, hi - 1, 2, v, beta);
            at(A, n, hi, hi - 2) = 0.0;
        }
    }
    // clean below the first subdiagonal
    for (int j = 0; j < n; ++j)
        for (int i = j + 2; i < n; ++i) at(A, n, i, j) = 0.0;
    return 0;
}

std::vector<cd> schur_eigenvalues(int n, const double* T) {
    std::vector<cd> ev(n);
    int i = 0;
    while (i < n) {
        if (i + 1 < n && at(T, n, i + 1, i) != 0.0) {
            const double a = at(T, n, i, i), b = at(T, n, i, i + 1);
            const double c = at(T, n, i + 1, i), d = at(T, n, i + 1, i + 1);
            const double p = 0.5 * (a - d);
            const double disc = p * p + b * c;
            const double m = 0.5 * (a + d);
            if (disc < 0.0) {
                const double im = std::sqrt(-disc);
                ev[i] = cd(m, im);
                ev[i + 1] = cd(m, -im);
            } else {
                const double sq = std::sqrt(disc);
                ev[i] = cd(m + sq, 0.0);
                ev[i + 1] = cd(m - sq, 0.0);
            }
            i += 2;
        } else {
            ev[i] = cd(at(T, n, i, i), 0.0);
            i += 1;
        }
    }
    return ev;
}

std::vector<cd> schur_eigenvector(int n, const double* T, const double* Z, int k, cd lambda) {
    std::vector<cd> x(n, cd(0.0, 0.0));
    const double tnorm = std::max(norm1_est(n, T), std::numeric_limits<double>::min());
    const double small = kEps * tnorm;
    int top;   // last index of the eigen-block
    if (k + 1 < n && at(T, n, k + 1, k) != 0.0) {
        const double a = at(T, n, k, k), b = at(T, n, k, k + 1);
        const double c = at(T, n, k + 1, k), d = at(T, n, k + 1, k + 1);
        cd x0 = b, x1 = lambda - a;
        const cd y0 = lambda - d, y1 = c;
        if (std::abs(x0) + std::abs(x1) < std::abs(y0) + std::abs(y1)) {
            x0 = y0;
            x1 = y1;
        }
        x[k] = x0;
        x[k + 1] = x1;
        top = k + 1;
    } else {
        x[k] = 1.0;
        top = k;
    }
    int i = k - 1;
    while (i >= 0) {
        if (i >= 1 && at(T, n, i, i - 1) != 0.0) {
            // 2x2 block at rows i-1, i
            cd r0 = 0.0, r1 = 0.0;
            for (int l = i + 1; l <= top; ++l) {
                r0 += at(T, n, i - 1, l) * x[l];
                r1 += at(T, n, i, l) * x[l];
            }
            const cd a = at(T, n, i - 1, i - 1) - lambda, b = at(T, n, i - 1, i);
            const cd c = at(T, n, i, i - 1), d = at(T, n, i, i) - lambda;
            cd det = a * d - b * c;
            if (std::abs(det) < small * small) det = small * small;
            x[i - 1] = (-r0 * d + b * r1) / det;
            x[i] = (-a * r1 + c * r0) / det;
            i -= 2;
        } else {
            cd r = 0.0;
            for (int l = i + 1; l <= top; ++l) r += at(T, n, i, l) * x[l];
            cd den = at(T, n, i, i) - lambda;
            if (std::abs(den) < small) den = small;
            x[i] = -r / den;
            i -= 1;
        }
    }
    std::vector<cd> y(n, cd(0.0, 0.0));
    for (int l = 0; l <= top; ++l) {
        if (x[l] == cd(0.0, 0.0)) continue;
        for (int r = 0; r < n; ++r) y[r] += at(Z, n, r, l) * x[l];
    }
    double nrm = 0.0;
    for (int r = 0; r < n; ++r) nrm += std::norm(y[r]);
    nrm = std::sqrt(nrm);
    if (nrm > 0)
        for (int r = 0; r < n; ++r) y[r] /= nrm;
    return y;
}

namespace {

// Solve the (pq) x (pq) system K u = rhs by Gaussian elimination with
// complete pivoting; returns false when K is numerically singular.
bool solve_small(int N, double* K, double* rhs, double* u) {
    int perm[4] = {0, 1, 2, 3};
    const double scale = [&] {
        double m = 0.0;
        for (int i = 0; i < N * N; ++i) m = std::max(m, std::fabs(K[i]));
        return m;
    }();
    if (scale == 0.0) return false;
    for (int c = 0; c < N; ++c) {
        int pr = c, pc = c;
        double best = -1;
        for (int i = c; i < N; ++i)
            for (int j = c; j < N; ++j)
                if (std::fabs(K[i * N + j]) > best) {
                    best = std::fabs(K[i * N + j]);
                    pr = i;
                    pc = j;
                }
        if (best <= 1e-14 * scale) return false;
        if (pr != c) {
            for (int j = 0; j < N; ++j) std::swap(K[pr * N + j], K[c * N + j]);
            std::swap(rhs[pr], rhs[c]);
        }
        if (pc != c) {
            for (int i = 0; i < N; ++i) std::swap(K[i * N + pc], K[i * N + c]);
            std::swap(perm[pc], perm[c]);
        }
        for (int i = c + 1; i < N; ++i) {
            const double f = K[i * N + c] / K[c * N + c];
            for (int j = c; j < N; ++j) K[i * N + j] -= f * K[c * N + j];
            rhs[i] -= f * rhs[c];
        }
    }
    double sol[4];
    for (int i = N - 1; i >= 0; --i) {
        double s = rhs[i];
        for (int j = i + 1; j < N; ++j) s -= K[i * N + j] * sol[j];
        sol[i] = s / K[i * N + i];
    }
    for (int i = 0; i < N; ++i) u[perm[i]] = sol[i];
    return true;
}

// Swap the adjacent diagonal blocks A11 (p x p, at row k) and A22 (q x q).
bool swap_blocks(int n, double* T, double* Z, int k, int p, int q) {
    const int N = p * q;
    double K[16] = {0}, rhs[4], u[4];
    // A11 X - X A22 = A12, X p x q, unknown X(i, j) at index i + j p
    for (int j = 0; j < q; ++j)
        for (int i = 0; i < p; ++i) {
            const int r = i + j * p;
            for (int l = 0; l < p; ++l) K[r * N + (l + j * p)] += at(T, n, k + i, k + l);
            for (int mm = 0; mm < q; ++mm) K[r * N + (i + mm * p)] -= at(T, n, k + p + mm, k + p + j);
            rhs[r] = at(T, n, k + i, k + p + j);
        }
    if (!solve_small(N, K, rhs, u)) return false;
    // QR of M = [X; -I_q] ((p+q) x q) with q Householder reflections
    const int L = p + q;
    double M[4][2];
    for (int j = 0; j < q; ++j) {
        for (int i = 0; i < p; ++i) M[i][j] = u[i + j * p];
        for (int i = 0; i < q; ++i) M[p + i][j] = (i == j) ? -1.0 : 0.0;
    }
    double vs[2][4], betas[2];
    for (int j = 0; j < q; ++j) {
        double x[4];
        const int len = L - j;
        for (int i = 0; i < len; ++i) x[i] = M[j + i][j];
        house(x, len, vs[j], &betas[j]);
        // apply to remaining columns of M
        for (int c = j; c < q; ++c) {
            double s = 0.0;
            for (int i = 0; i < len; ++i) s += vs[j][i] * M[j + i][c];
            s *= betas[j];
            for (int i = 0; i < len; ++i) M[j + i][c] -= s * vs[j][i];
        }
    }
    // T <- Q^T T Q and Z <- Z Q with Q = H_0 H_1 ...
    for (int j = 0; j < q; ++j) {
        const int len = L - j;
        apply_left(n, T, k + j, len, k, n - 1, vs[j], betas[j]);
        apply_right(n, T, 0, std::min(n - 1, k + L - 1), k + j, len, vs[j], betas[j]);
        apply_right(n, Z, 0, n - 1, k + j, len, vs[j], betas[j]);
    }
    // the new (p x q) lower-left block and everything below the first
    // subdiagonal of the swapped rows are zero up to rounding
    for (int j = k; j < k + q; ++j)
        for (int i = k + q; i < k + L; ++i) at(T, n, i, j) = 0.0;
    for (int j = k; j < k + L; ++j)
        for (int i = j + 2; i < k + L; ++i) at(T, n, i, j) = 0.0;
    if (q == 2) standardize_2x2(n, T, Z, k);
    if (p == 2) standardize_2x2(n, T, Z, k + q);
    return true;
}

}  // namespace

int schur_reorder(int n, double* T, double* Z, const std::function<bool(cd)>& wanted) {
    auto block_size = [&](int i) { return (i + 1 < n && at(T, n, i + 1, i) != 0.0) ? 2 : 1; };
    int ks = 0;
    int i = 0;
    while (i < n) {
        const int s = block_size(i);
        const std::vector<cd> ev = schur_eigenvalues(n, T);
        if (wanted(ev[i])) {
            int pos = i, sz = s;
            while (pos > ks) {
                const int sa = (pos >= 2 && at(T, n, pos - 1, pos - 2) != 0.0) ? 2 : 1;
                if (!swap_blocks(n, T, Z, pos - sa, sa, sz)) return -1;
                pos -= sa;
                sz = block_size(pos);
            }
            ks += sz;
            i += s;
        } else {
            i += s;
        }
    }
    return ks;
}

}  // namespace dense
}  // namespace nsstab
