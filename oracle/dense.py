"""Oracle: explicit assembly of the operators by columns (TEST INFRASTRUCTURE ONLY).

Only feasible on small grids (n = nx ny up to a few thousand).  The paper
notes that assembling A or M is impractical at scale (Sec. 3); here the dense
matrices serve to pin the matrix-free solvers on small cases.
"""
from __future__ import annotations

import numpy as np

from . import ns2d


def _columns(op, cfg: ns2d.Config, batch: int = 256):
    n = cfg.n
    out = np.zeros((n, n))
    for c0 in range(0, n, batch):
        c1 = min(n, c0 + batch)
        E = np.zeros((c1 - c0, cfg.ny, cfg.nx))
        E.reshape(c1 - c0, n)[np.arange(c1 - c0), np.arange(c0, c1)] = 1.0
        out[:, c0:c1] = op(E).reshape(c1 - c0, n).T
    return out


def assemble_M(base: ns2d.Base, T: float, cfg: ns2d.Config) -> np.ndarray:
    """Dense M = exp(T A) as realised by the stepper (Eq. 42), column by column."""
    return _columns(lambda E: ns2d.apply_expTL(base, E, T, cfg), cfg)


def assemble_A(base: ns2d.Base, cfg: ns2d.Config) -> np.ndarray:
    """Dense semi-discrete linearised operator A (Eq. 30) of this discretisation."""
    return _columns(lambda E: ns2d.semidiscrete_linear_rhs(E, base, cfg), cfg)
