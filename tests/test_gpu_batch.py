"""Batched stepping: every member of a batch (its own Reynolds number and
cylinder diameter, its own base flow) matches the FP64 oracle run alone, and
the lockstep batched eigen-solver matches per-member dense eigendecompositions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, krylov, ns2d, sfd  # noqa: E402
from paper_1804_03859_gb300 import inputs, nsstab  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _match(a, b):
    return max(np.min(np.abs(b - x)) for x in a)


RES = [40.0, 60.0, 100.0]
DS = [0.8, 1.0, 1.2]


def _member_cfg(nx, ny, k, dt):
    return ns2d.Config(nx=nx, ny=ny, dt=dt, Re=RES[k], cyl_D=DS[k])


@pytest.mark.parametrize("nx,ny,per_set", [(64, 32, 2), (128, 64, 1), (256, 128, 3)])
def test_batched_nonlinear_and_linear_steps_match_each_member(nx, ny, per_set):
    dt = 0.01 * 128 / nx
    st = nsstab.Stepper(nx=nx, ny=ny, dt=dt, Re=RES, cyl_D=DS, per_set=per_set)
    B = 3 * per_set
    assert (st.members, st.sets) == (B, 3)
    w0 = np.stack([inputs.wake_like_field(ny, nx, seed=30 + m) for m in range(B)])
    t = _dev(w0)
    st.step_nonlinear(t, 3)
    got = _host(t)
    for m in range(B):
        ref = ns2d.step_nonlinear(w0[m], 3, _member_cfg(nx, ny, m // per_set, dt))
        assert _rel(got[m], ref) <= 3e-12, m
    bases = np.stack([inputs.wake_like_field(ny, nx, seed=40 + k) for k in range(3)])
    v = np.stack([inputs.gaussian_field(ny, nx, seed=50 + m) for m in range(B)])
    out = torch.empty(B, ny, nx, dtype=torch.float64, device="cuda")
    st.apply_expTL(_dev(bases), _dev(v), out, 5 * dt)
    got = _host(out)
    for m in range(B):
        c = _member_cfg(nx, ny, m // per_set, dt)
        ref = ns2d.apply_expTL(ns2d.Base.from_omega(bases[m // per_set], c), v[m], 5 * dt, c)
        assert _rel(got[m], ref) <= 5e-12, m
    r = st.stepper_residual(_dev(w0))
    for m in range(B):
        rr = ns2d.residual(w0[m], _member_cfg(nx, ny, m // per_set, dt))
        assert abs(r[m] - rr) <= 1e-11 * rr


def test_batched_poisson_and_long_graph_runs():
    nx, ny = 64, 32
    st = nsstab.Stepper(nx=nx, ny=ny, dt=0.02, Re=RES, cyl_D=DS)
    w = np.stack([inputs.gaussian_field(ny, nx, seed=60 + m) for m in range(3)])
    psi = torch.empty(3, ny, nx, dtype=torch.float64, device="cuda")
    st.stepper_poisson(_dev(w), psi)
    got = _host(psi)
    for m in range(3):
        assert _rel(got[m], ns2d.streamfunction(w[m], _member_cfg(nx, ny, m, 0.02))) <= 1e-13
    t = torch.zeros(3, ny, nx, dtype=torch.float64, device="cuda")
    st.step_nonlinear(t, 300)
    got = _host(t)
    for m in range(3):
        ref = ns2d.step_nonlinear(np.zeros((ny, nx)), 300, _member_cfg(nx, ny, m, 0.02))
        assert _rel(got[m], ref) <= 300 * 1e-12


def test_batched_sfd_converges_every_member():
    nx, ny = 32, 16
    Re = [15.0, 20.0]
    st = nsstab.Stepper(nx=nx, ny=ny, dt=0.02, Re=Re)
    t = torch.zeros(2, ny, nx, dtype=torch.float64, device="cuda")
    rc, r, steps = st.sfd_baseflow(t, chi=0.5, Delta=1.0, tol=1e-10, max_steps=40000, check_every=200)
    assert rc == nsstab.OK and np.all(r <= 1e-10)
    got = _host(t)
    for k in range(2):
        c = ns2d.Config(nx=nx, ny=ny, dt=0.02, Re=Re[k])
        assert ns2d.residual(got[k], c) <= 2e-10


def test_batched_eigs_match_dense_per_member():
    nx, ny, T = 32, 16, 2.0
    Re = [50.0, 40.0]
    per_set = 2
    bases = np.stack([inputs.wake_like_field(ny, nx, seed=7), inputs.wake_like_field(ny, nx, seed=8)])
    dense_mu = []
    for k in range(2):
        c = ns2d.Config(nx=nx, ny=ny, dt=0.02, Re=Re[k])
        M = dense.assemble_M(ns2d.Base.from_omega(bases[k], c), T, c)
        mu = np.linalg.eigvals(M)
        dense_mu.append(mu[krylov.leading_order(mu)])
    st = nsstab.Stepper(nx=nx, ny=ny, dt=0.02, Re=Re, per_set=per_set)
    v0 = np.stack([inputs.gaussian_field(ny, nx, seed=70 + m) for m in range(4)])
    # plain Arnoldi (one factorisation) and Krylov-Schur with restarts
    for m_dim, restarts, tol in ((150, 0, 1e-10), (40, 200, 1e-11)):
        res = st.batch_arnoldi_eigs(_dev(bases), _dev(v0), m=m_dim, nev=4, tol=tol, T=T, max_restarts=restarts)
        assert len(res) == 4
        for m, r in enumerate(res):
            assert r.n_conv == len(r.mu), (m, m_dim)
            assert _match(r.mu, dense_mu[m // per_set][:6]) <= 1e-10, (m, m_dim)
        if restarts:
            assert any(r.n_matvec > m_dim for r in res)


def test_single_arnoldi_still_rejects_batches():
    st = nsstab.Stepper(nx=16, ny=8, Re=[40.0, 50.0])
    v0 = torch.zeros(2, 8, 16, dtype=torch.float64, device="cuda")
    with pytest.raises((nsstab.NsstabError, ValueError)):
        st.arnoldi_eigs(None, v0, m=4, nev=1, tol=1e-8, T=0.5)
