// Small dense FP64 eigen-solver on the host for the Krylov layer: the
// Hessenberg / Schur eigensolve of the projected matrix (Sec. 3.2.1, the
// Ritz pairs of H_m) and the ordered real Schur form of the Krylov-Schur
// restart (Sec. 3.2.2, step 3).  Matrices are column-major, a(i, j) at
// a[i + j * n].
#pragma once

#include <complex>
#include <functional>
#include <vector>

namespace nsstab {
namespace dense {

using cd = std::complex<double>;

// A <- Q^T A Q upper Hessenberg by Householder reflections; Q <- Q * Q_H.
void hessenberg(int n, double* A, double* Q);

// A (upper Hessenberg) <- T = Z^T A Z in real Schur form (2x2 diagonal
// blocks only for complex-conjugate pairs), Z <- Z * (accumulated rotations),
// by the implicit double-shift (Francis) QR iteration.  Returns 0, or -1 if
// the iteration did not converge.
int schur(int n, double* A, double* Z);

// Eigenvalues of the quasi-triangular T, in diagonal order.
std::vector<cd> schur_eigenvalues(int n, const double* T);

// Unit-norm eigenvector y = Z x of Z T Z^T for the eigenvalue lambda of the
// diagonal block starting at row k (lambda with Im >= 0 for a 2x2 block).
std::vector<cd> schur_eigenvector(int n, const double* T, const double* Z, int k, cd lambda);

// Reorder T, Z so that the blocks whose eigenvalue satisfies `wanted` come
// first (relative order kept).  Returns the dimension of the wanted leading
// block, or -1 if a swap was too ill-conditioned to perform.
int schur_reorder(int n, double* T, double* Z, const std::function<bool(cd)>& wanted);

}  // namespace dense
}  // namespace nsstab
