"""Oracle: Newton-Krylov fixed-point solver (TEST INFRASTRUCTURE ONLY).

Newton iteration of Sec. 3.1.2 (Eq. 43): x_{k+1} = x_k - (I - M)^{-1}
(x_k - G(x_k)), M the Jacobian of the map G (Eq. 42).  The (n x n) solve
is left to a Krylov method; here restarted GMRES with CGS2 Arnoldi
(Algorithm 1) and Givens rotations, the projected least-squares problem
solved by back substitution.  For the Navier-Stokes map G = Phi_T (T/dt
steps of the nonlinear stepper) the product with M is, by default, the exact
discrete tangent (ns2d.apply_tangent: the linearised step about each point
of the trajectory, advanced together with it); jacobian="frozen" instead
marches the linearised equations about the current iterate, which equals
the exact Jacobian at a steady state and differs from it by O(||x - G(x)||)
near one.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import ns2d


def gmres(matvec, b, m: int, rtol: float, max_restarts: int = 0):
    """Solve A x = b by GMRES(m) from x = 0.  Returns (x, relative residual, products)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    n = b.size
    x = np.zeros(n)
    beta0 = np.linalg.norm(b)
    if beta0 == 0.0:
        return x, 0.0, 0
    nmv = 0
    r = b.copy()
    rel = 1.0
    for _ in range(max_restarts + 1):
        beta = np.linalg.norm(r)
        V = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            w = matvec(V[:, j])
            nmv += 1
            Vj = V[:, : j + 1]
            h1 = Vj.T @ w
            w = w - Vj @ h1
            h2 = Vj.T @ w
            w = w - Vj @ h2
            h = h1 + h2
            hn = np.linalg.norm(w)
            # previous rotations on the new column
            for i in range(j):
                t = cs[i] * h[i] + sn[i] * h[i + 1]
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1]
                h[i] = t
            d = np.hypot(h[j], hn)
            cs[j], sn[j] = (1.0, 0.0) if d == 0.0 else (h[j] / d, hn / d)
            h[j] = d
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            H[: j + 1, j] = h
            k = j + 1
            rel = abs(g[j + 1]) / beta0
            if rel <= rtol or hn == 0.0:
                break
            V[:, j + 1] = w / hn
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + V[:, :k] @ y
        if rel <= rtol:
            break
        r = b - matvec(x)
        nmv += 1
        rel = np.linalg.norm(r) / beta0
        if rel <= rtol:
            break
    return x, rel, nmv


@dataclasses.dataclass
class NewtonResult:
    x: np.ndarray
    residual: float
    iters: int
    matvecs: int
    converged: bool


def newton_krylov(G, jac_matvec, residual, x0, tol: float, max_newton: int, m: int = 50,
                  gmres_rtol: float = 1e-3, max_restarts: int = 2) -> NewtonResult:
    """Newton iteration of Eq. 43 with GMRES(m) for (I - M) dx = x - G(x).

    G: the map; jac_matvec(x, v): M v at x; residual(x): the stopping measure.
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    shape = x.shape
    nmv = 0
    for k in range(max_newton + 1):
        res = residual(x)
        if res <= tol:
            return NewtonResult(x, res, k, nmv, True)
        if k == max_newton:
            break
        r = (x - G(x)).ravel()
        A = lambda v: v - jac_matvec(x, v.reshape(shape)).ravel()
        dx, _, n = gmres(A, r, m, gmres_rtol, max_restarts)
        nmv += n
        x = x - dx.reshape(shape)
    return NewtonResult(x, residual(x), max_newton, nmv, False)


def newton_baseflow(cfg: ns2d.Config, omega0, T: float, tol: float, max_newton: int, m: int = 50,
                    gmres_rtol: float = 1e-3, max_restarts: int = 2, jacobian: str = "tangent") -> NewtonResult:
    """Steady base flow: fixed point of Phi_T (T/dt nonlinear steps), stopped on
    the residual r(q) = ||G_1(q) - q||_h / dt."""
    nT = ns2d.steps_per_period(T, cfg)
    G = lambda q: ns2d.step_nonlinear(q, nT, cfg)
    if jacobian == "tangent":
        J = lambda q, v: ns2d.apply_tangent(q, v, T, cfg)
    else:
        J = lambda q, v: ns2d.apply_expTL(ns2d.Base.from_omega(q, cfg), v, T, cfg)
    return newton_krylov(G, J, lambda q: ns2d.residual(q, cfg), omega0, tol, max_newton, m, gmres_rtol,
                         max_restarts)
