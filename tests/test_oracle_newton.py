"""Pins of the oracle Newton-Krylov solver (Sec. 3.1.2, Eq. 43)."""
import json
import os

import numpy as np
import scipy.sparse.linalg

from oracle import newton, ns2d, sfd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gmres_solves_a_nonsymmetric_system_like_scipy():
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, rel, nmv = newton.gmres(lambda v: A @ v, b, m=60, rtol=1e-12)
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    # restarted: GMRES(5) with restarts still converges on this well-conditioned system
    x5, rel5, _ = newton.gmres(lambda v: A @ v, b, m=5, rtol=1e-10, max_restarts=100)
    assert rel5 <= 1e-10 and np.linalg.norm(x5 - xs) <= 1e-8 * np.linalg.norm(xs)


def test_newton_finds_all_three_duffing_fixed_points():
    """Unlike SFD, Newton converges to the saddle as well (Sec. 3.1.2 vs 3.1.1)."""
    spec = json.load(open(os.path.join(GOLDEN, "duffing.json")))
    d = spec["damping"]
    dt = 0.01

    def G(X):
        x, y = X
        return X + dt * np.array([y, -d * y + x - x ** 3])

    def J(X, v):
        x, _ = X
        return v + dt * np.array([v[1], -d * v[1] + (1 - 3 * x * x) * v[0]])

    for p, start in zip(spec["fixed_points"], ([0.2, 0.1], [0.8, -0.2], [-1.3, 0.2])):
        res = newton.newton_krylov(G, J, lambda X: np.linalg.norm(G(X) - X) / dt, np.array(start),
                                   tol=1e-12, max_newton=30, m=2, gmres_rtol=1e-14)
        assert res.converged
        assert np.allclose(res.x, [p["x"], p["y"]], atol=1e-10)


def test_newton_base_flow_matches_sfd_and_meets_the_residual_target():
    cfg = ns2d.Config(nx=32, ny=16, dt=0.02, Re=20.0)
    res = newton.newton_baseflow(cfg, np.zeros((16, 32)), T=0.4, tol=1e-10, max_newton=20, m=40)
    assert res.converged and res.residual <= 1e-10
    assert res.iters <= 10
    X, r, steps, ok = sfd.sfd_baseflow(cfg, np.zeros((16, 32)), 0.5, 1.0, tol=1e-11, max_steps=60000,
                                       check_every=200)
    assert ok
    assert np.abs(res.x - X).max() <= 1e-8 * np.abs(X).max()


def test_exact_tangent_and_frozen_jacobian_reach_the_same_fixed_point():
    """The default Newton Jacobian is the co-integrated tangent; the frozen
    linearisation reaches the same fixed point (it is exact there) but
    needs at least as many iterations from a start far from it."""
    cfg = ns2d.Config(nx=32, ny=16, dt=0.02, Re=40.0)
    q0 = ns2d.step_nonlinear(np.zeros((16, 32)), 20, cfg)
    a = newton.newton_baseflow(cfg, q0, T=0.4, tol=1e-10, max_newton=30, m=40, gmres_rtol=1e-8)
    b = newton.newton_baseflow(cfg, q0, T=0.4, tol=1e-10, max_newton=30, m=40, gmres_rtol=1e-8,
                               jacobian="frozen")
    assert a.converged and b.converged
    assert np.abs(a.x - b.x).max() <= 1e-8 * np.abs(a.x).max()
    assert a.iters <= b.iters
