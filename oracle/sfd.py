"""Oracle: selective frequency damping (TEST INFRASTRUCTURE ONLY).

Eq. 40 (Sec. 3.1.1): dX/dt = F(X) - chi (X - Y),  dY/dt = (X - Y)/Delta.

Time discretisation (a reading; the paper leaves it to the host code): one
step of the plain time-stepper X* = G(X^n) is followed by an explicit Euler
step of the two forcing terms evaluated at (X*, Y^n):
    X^{n+1} = X* - dt chi (X* - Y^n),   Y^{n+1} = Y^n + dt (X* - Y^n)/Delta.
At a fixed point X = Y = G(X), so the control vanishes (Sec. 3.1.1).
"""
from __future__ import annotations

import numpy as np

from . import ns2d


def sfd_forcing(Xs, Y, chi: float, Delta: float, dt: float):
    """Explicit Euler step of the SFD forcing terms of Eq. 40 at (X*, Y)."""
    return Xs - dt * chi * (Xs - Y), Y + dt * (Xs - Y) / Delta


def sfd_map(G, x0, chi: float, Delta: float, dt: float, nsteps: int):
    """SFD around a memoryless step map G (e.g. explicit Euler of a toy ODE).

    Returns the trajectory of X as an array of shape (nsteps + 1, n).
    """
    X = np.array(x0, dtype=np.float64, copy=True)
    Y = X.copy()
    traj = [X.copy()]
    for _ in range(nsteps):
        X, Y = sfd_forcing(G(X), Y, chi, Delta, dt)
        traj.append(X.copy())
    return np.array(traj)


def sfd_baseflow(cfg: ns2d.Config, omega0, chi: float, Delta: float, tol: float,
                 max_steps: int, check_every: int = 100):
    """March the SFD-controlled nonlinear stepper until r(X) <= tol.

    The Navier-Stokes part keeps its AB2 history across steps (AB1 on the
    first).  Every ``check_every`` steps the base-flow residual r(X) of
    ``ns2d.residual`` is evaluated.  Returns (X, r, steps, converged).
    """
    X = np.array(omega0, dtype=np.float64, copy=True)
    Y = X.copy()
    Nh = None
    r = np.inf
    for k in range(max_steps):
        Xs, Nh = ns2d.step(X, Nh, cfg, first=(k == 0))
        X, Y = sfd_forcing(Xs, Y, chi, Delta, cfg.dt)
        if (k + 1) % check_every == 0 or k + 1 == max_steps:
            r = ns2d.residual(X, cfg)
            if r <= tol:
                return X, r, k + 1, True
    return X, r, max_steps, False
