"""Pins of the oracle Krylov solvers, SFD and dense assembly.

The eigen-solvers are checked against LAPACK's dense eigendecomposition of the
explicitly assembled propagator, against the toy systems the paper prints
(golden fixtures under tests/golden, each with its citation), and against
identities that any Arnoldi factorisation satisfies (Eqs. 57 and 63).
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import dense, krylov, ns2d, sfd
from paper_1804_03859_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _match(a, b):
    """Max distance from each value of a to the nearest value of b."""
    return max(np.min(np.abs(b - x)) for x in a)


@pytest.fixture(scope="module")
def small_case():
    cfg = ns2d.Config(nx=32, ny=16, dt=0.02, Re=50.0)
    base = ns2d.Base.from_omega(inputs.wake_like_field(16, 32, seed=7), cfg)
    # T = 2 spreads the clustered moduli of this advection-dominated spectrum
    # enough for a plain Arnoldi factorisation of order 150 to converge
    T = 2.0
    M = dense.assemble_M(base, T, cfg)
    mu = np.linalg.eigvals(M)
    return cfg, base, T, M, mu[krylov.leading_order(mu)]


def test_schmid_toy_eigenvalues():
    spec = json.load(open(os.path.join(GOLDEN, "schmid_toy.json")))
    T = 2.0
    for case in spec["cases"]:
        A = np.array(case["A"])
        lam = np.array(case["lambda"])
        Re = case["Re"]
        assert np.allclose(np.diag(A), [1 / 100 - 1 / Re, -2 / Re])
        M = scipy.linalg.expm(A * T)
        res = krylov.arnoldi_eigs(lambda x: M @ x, np.array([1.0, 0.3]), m=2, nev=2, tol=1e-12)
        got = np.sort(np.log(res.mu.real) / T)
        assert np.allclose(got, np.sort(lam), atol=1e-12)
        assert (np.abs(res.mu).max() < 1.0) == case["stable"]


def test_dense_eig_matches_arnoldi(small_case):
    cfg, base, T, M, mu_dense = small_case
    v0 = inputs.gaussian_field(cfg.ny, cfg.nx, seed=11).ravel()
    res = krylov.arnoldi_eigs(lambda x: M @ x, v0, m=150, nev=4, tol=1e-10)
    assert res.n_conv == res.mu.size
    assert _match(res.mu, mu_dense[:8]) < 1e-12


def test_arnoldi_relation_orthogonality_and_residual_estimate(small_case):
    cfg, base, T, M, _ = small_case
    m = 40
    v0 = inputs.gaussian_field(cfg.ny, cfg.nx, seed=12).ravel()
    V, H, j = krylov.arnoldi(lambda x: M @ x, v0, m)
    assert j == m
    assert np.abs(V.T @ V - np.eye(m + 1)).max() < 1e-13
    # Eq. 57: M V_m = V_{m+1} H
    assert np.linalg.norm(M @ V[:, :m] - V @ H) < 1e-12 * np.linalg.norm(M, 2)
    b = np.zeros(m)
    b[-1] = H[m, m - 1]
    mu, Y, res = krylov.ritz(H[:m, :m], b)
    # Eq. 63: the true residual of each Ritz pair equals |beta e_m^T y|
    for k in range(m):
        x = V[:, :m] @ Y[:, k]
        true = np.linalg.norm(M @ x - mu[k] * x)
        assert abs(true - res[k]) < 1e-11


def test_arnoldi_through_the_stepper_matches_dense(small_case):
    """The matrix-free matvec (time marching) gives the dense spectrum."""
    cfg, base, T, M, mu_dense = small_case
    mv = lambda x: ns2d.apply_expTL(base, x.reshape(cfg.ny, cfg.nx), T, cfg).ravel()
    v0 = inputs.gaussian_field(cfg.ny, cfg.nx, seed=13).ravel()
    res = krylov.arnoldi_eigs(mv, v0, m=150, nev=4, tol=1e-10)
    assert res.n_conv == res.mu.size
    assert _match(res.mu, mu_dense[:6]) < 1e-12


def test_krylov_schur_matches_dense(small_case):
    cfg, base, T, M, mu_dense = small_case
    v0 = inputs.gaussian_field(cfg.ny, cfg.nx, seed=14).ravel()
    res = krylov.krylov_schur(lambda x: M @ x, v0, m=40, nev=4, tol=1e-11, max_restarts=200)
    assert res.n_conv == res.mu.size and res.restarts > 0
    assert _match(res.mu, mu_dense[:6]) < 1e-11
    # matvec count: m for the first factorisation, then m - p per restart
    assert res.n_matvec > 40


def test_log_mu_over_T_converges_to_eig_A_first_order():
    """mu = exp(lambda T) up to the O(dt) splitting error (Eq. 42)."""
    cfg = ns2d.Config(nx=32, ny=16, Re=50.0, eta=0.05)
    base = ns2d.Base.from_omega(inputs.wake_like_field(16, 32, seed=5), cfg)
    A = dense.assemble_A(base, cfg)
    lam = np.linalg.eigvals(A)
    lam = lam[np.abs(lam) > 1e-9]
    lam_lead = lam[np.argsort(-lam.real)][:4]
    T = 0.4
    errs = []
    for dt in (0.02, 0.01, 0.005):
        cfg.dt = dt
        M = dense.assemble_M(base, T, cfg)
        mu = np.linalg.eigvals(M)
        mu = mu[np.abs(mu) > 1e-12]
        lt = np.log(mu.astype(complex)) / T
        errs.append(max(np.min(np.abs(lt - l)) for l in lam_lead))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert errs[-1] < 1e-2
    assert 1.6 < r1 < 2.5 and 1.6 < r2 < 2.5, errs


def _duffing_G(dt, d):
    def G(X):
        x, y = X
        return X + dt * np.array([y, -d * y + x - x ** 3])
    return G


def test_sfd_cannot_stabilise_the_duffing_saddle():
    spec = json.load(open(os.path.join(GOLDEN, "duffing.json")))
    d = spec["damping"]
    dt = 0.01
    G = _duffing_G(dt, d)
    fps = {(p["x"], p["y"]): p["kind"] for p in spec["fixed_points"]}
    for (x, y), kind in fps.items():
        F = G(np.array([x, y])) - np.array([x, y])
        assert np.allclose(F, 0.0)
    # start next to the saddle: SFD leaves it (real unstable eigenvalue)
    traj = sfd.sfd_map(G, [1e-3, 0.0], chi=1.0, Delta=1.0, dt=dt, nsteps=20000)
    end = traj[-1]
    assert np.hypot(*end) > 0.5
    assert min(np.hypot(end[0] - 1, end[1]), np.hypot(end[0] + 1, end[1])) < 1e-3
    # start near a stable spiral: SFD converges to it
    traj = sfd.sfd_map(G, [0.7, 0.2], chi=1.0, Delta=1.0, dt=dt, nsteps=20000)
    assert np.hypot(traj[-1][0] - 1, traj[-1][1]) < 1e-6


def test_sfd_closed_loop_rate_matches_the_quadratic():
    """For dX/dt = lambda X (oscillatory, unstable), Eq. 40 has eigenvalues s with
    (s - lambda + chi)(s + 1/Delta) = chi/Delta."""
    a, w = 0.05, 1.0
    Amat = np.array([[a, -w], [w, a]])
    chi, Delta, dt = 0.5, 1.0, 1e-3
    G = lambda X: X + dt * Amat @ X
    traj = sfd.sfd_map(G, [1.0, 0.0], chi, Delta, dt, nsteps=60000)
    nrm = np.linalg.norm(traj, axis=1)
    t = dt * np.arange(traj.shape[0])
    sl = slice(30000, 60000)
    rate = np.polyfit(t[sl], np.log(nrm[sl]), 1)[0]
    lam = a + 1j * w
    s = np.roots([1.0, (1 / Delta) + chi - lam, (chi - lam) / Delta - chi / Delta])
    assert rate < 0
    assert abs(rate - s.real.max()) < 5e-3


def test_sfd_reaches_a_steady_base_flow():
    cfg = ns2d.Config(nx=32, ny=16, dt=0.02, Re=20.0)
    X, r, steps, ok = sfd.sfd_baseflow(cfg, np.zeros((16, 32)), chi=0.5, Delta=1.0,
                                       tol=1e-10, max_steps=40000, check_every=200)
    assert ok, (r, steps)
    assert ns2d.residual(X, cfg) <= 1e-10
    mirror = X[(-np.arange(16)) % 16, :]
    assert np.abs(X + mirror).max() <= 1e-9 * np.abs(X).max()
