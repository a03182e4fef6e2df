"""Oracle: Krylov eigenvalue solvers (TEST INFRASTRUCTURE ONLY).

* ``arnoldi``      - Algorithm 1 (m-step Arnoldi factorisation, Sec. 3.2.1),
                     M V_m = V_m H_m + r_m e_m^T (Eq. 57), with a second
                     classical Gram-Schmidt pass (CGS2) after each product.
* ``ritz``         - Ritz pairs of H_m and the residual |beta e_m^T y| of Eq. 63.
* ``krylov_schur`` - the expansion / Schur-sort / truncation / re-expansion
                     cycle of Sec. 3.2.2 (Eqs. 60-63).

The matrix-vector product is any callable x -> M x on flat float64 vectors.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg


def _cgs2(Vj: np.ndarray, w: np.ndarray):
    """Classical Gram-Schmidt against the columns of Vj, applied twice."""
    h1 = Vj.T @ w
    w = w - Vj @ h1
    h2 = Vj.T @ w
    w = w - Vj @ h2
    return h1 + h2, w


def arnoldi(matvec, v0: np.ndarray, m: int, V=None, H=None, start: int = 0):
    """Algorithm 1 with CGS2.  Returns (V, H, j_done).

    V is n x (m+1) with orthonormal columns, H is (m+1) x m upper Hessenberg
    (or, when restarting from a Krylov-Schur decomposition of order ``start``,
    H holds that decomposition in its leading (start+1) x start block).  The
    loop stops early on an exact invariant subspace (beta == 0); ``j_done`` is
    the number of columns of H that were filled.
    """
    if V is None:
        v0 = np.asarray(v0, dtype=np.float64).ravel()
        n = v0.size
        V = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        V[:, 0] = v0 / np.linalg.norm(v0)
    for j in range(start, m):
        w = np.asarray(matvec(V[:, j]), dtype=np.float64).ravel()
        h, w = _cgs2(V[:, : j + 1], w)
        H[: j + 1, j] = h
        beta = np.linalg.norm(w)
        H[j + 1, j] = beta
        if beta == 0.0:
            return V, H, j + 1
        V[:, j + 1] = w / beta
    return V, H, m


def ritz(B: np.ndarray, b: np.ndarray):
    """Ritz pairs of the order-m Krylov decomposition M V = V B + v b^T.

    Returns (mu, Y, res): eigenvalues of B, unit-norm eigenvectors (columns of
    Y) and residuals |b^T y| (Eq. 63; b = beta e_m for an Arnoldi factorisation).
    """
    mu, Y = np.linalg.eig(B)
    Y = Y / np.linalg.norm(Y, axis=0, keepdims=True)
    res = np.abs(b @ Y)
    return mu, Y, res


def leading_order(mu: np.ndarray) -> np.ndarray:
    """Indices sorting by |mu| descending, then Im(mu) descending."""
    return np.lexsort((-mu.imag, -np.abs(mu)))


def take_leading(mu: np.ndarray, nev: int) -> int:
    """Number of leading values to keep so that no conjugate pair is split."""
    order = leading_order(mu)
    k = min(nev, mu.size)
    if 0 < k < mu.size:
        last = mu[order[k - 1]]
        if last.imag > 0 and abs(mu[order[k]] - np.conj(last)) <= 1e-12 * max(1.0, abs(last)):
            k += 1
    return k


@dataclasses.dataclass
class EigResult:
    mu: np.ndarray          # leading Ritz values, |mu| descending
    residual: np.ndarray    # |b^T y| of each
    vectors: np.ndarray     # n x k complex Ritz vectors V y
    n_conv: int
    n_matvec: int
    restarts: int


def arnoldi_eigs(matvec, v0, m: int, nev: int, tol: float, want_vectors=False) -> EigResult:
    """m-step Arnoldi (no restart); leading nev Ritz pairs and residuals."""
    V, H, j = arnoldi(matvec, v0, m)
    b = np.zeros(j)
    b[j - 1] = H[j, j - 1]
    mu, Y, res = ritz(H[:j, :j], b)
    order = leading_order(mu)
    k = take_leading(mu, nev)
    sel = order[:k]
    vecs = V[:, :j] @ Y[:, sel] if want_vectors else None
    return EigResult(mu[sel], res[sel], vecs, int(np.sum(res[sel] <= tol)), j, 0)


def krylov_schur(matvec, v0, m: int, nev: int, tol: float, max_restarts: int = 50,
                 delta: float = 0.05, want_vectors=False) -> EigResult:
    """Krylov-Schur method of Sec. 3.2.2.

    1. order-m Arnoldi decomposition; 2. stop when the nev leading Ritz values
    have |b^T y| <= tol; 3. real Schur form B = Q S Q^T sorted so that the p
    wanted values come first; 4. truncate to order p:
    M (V Q_p) = (V Q_p) S_11 + v_{m+1} (b^T Q_p); 5. re-expand to order m
    orthogonalising against all kept vectors; repeat.

    Reading of the wanted set: the paper keeps |mu| >= 1 - delta; here p is
    that count clamped to [nev, m/2] (so that every restart both keeps the
    requested values and frees room to expand), then raised by one if the
    cut would split a complex-conjugate pair.
    """
    V, B, j = arnoldi(matvec, v0, m)
    n_matvec = j
    restarts = 0
    while True:
        b = B[m, :m].copy()
        mu, Y, res = ritz(B[:m, :m], b)
        order = leading_order(mu)
        k = take_leading(mu, nev)
        sel = order[:k]
        conv = int(np.sum(res[sel] <= tol))
        if conv >= k or restarts >= max_restarts or j < m:
            vecs = V[:, :m] @ Y[:, sel] if want_vectors else None
            return EigResult(mu[sel], res[sel], vecs, conv, n_matvec, restarts)
        # wanted set
        mags = np.abs(mu)
        p = int(np.sum(mags >= 1.0 - delta))
        p = max(k, min(p, m // 2))
        thr_mu = mu[order[p - 1]]
        if thr_mu.imag != 0.0 and p < m:
            # keep the conjugate partner of the last kept value
            partner = np.conj(thr_mu)
            rest = mu[order[p:]]
            if np.any(np.abs(rest - partner) <= 1e-12 * max(1.0, abs(thr_mu))):
                p += 1
        thr = np.sort(mags)[::-1][p - 1]
        S, Q, sdim = scipy.linalg.schur(
            B[:m, :m], output="real",
            sort=lambda re, im: np.hypot(re, im) >= thr * (1.0 - 1e-12))
        p = sdim
        Vp = V[:, :m] @ Q[:, :p]
        vnext = V[:, m].copy()
        b1 = b @ Q[:, :p]
        V[:, :p] = Vp
        V[:, p] = vnext
        V[:, p + 1:] = 0.0
        B[:] = 0.0
        B[:p, :p] = S[:p, :p]
        B[p, :p] = b1
        V, B, j = arnoldi(matvec, None, m, V=V, H=B, start=p)
        n_matvec += j - p
        restarts += 1
