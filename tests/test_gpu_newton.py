"""GPU Newton-Krylov base flow (Sec. 3.1.2, Eq. 43) against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import newton, ns2d  # noqa: E402
from paper_1804_03859_gb300 import inputs, nsstab  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("prec,tol", [(64, 1e-11), (48, 1e-11), (32, 2e-5)])
def test_tangent_matches_the_oracle_co_integration(prec, tol):
    kw = dict(nx=64, ny=32, dt=0.02, Re=50.0)
    cfg = ns2d.Config(**kw)
    q = inputs.wake_like_field(32, 64, seed=5)
    v = inputs.smooth_field(32, 64, seed=6)
    T = 10 * cfg.dt
    st = nsstab.Stepper(per_set=2, precision=prec, **kw)
    out = torch.empty(32, 64, dtype=torch.float64, device="cuda")
    st.apply_tangent(_dev(q), _dev(v), out, T)
    ref = ns2d.apply_tangent(q, v, T, cfg)
    got = out.cpu().numpy()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    # the frozen linearisation is a different operator away from a fixed point
    frozen = ns2d.apply_expTL(ns2d.Base.from_omega(q, cfg), v, T, cfg)
    assert np.linalg.norm(frozen - ref) > 1e2 * tol * np.linalg.norm(ref)


def test_tangent_through_graph_chunks_and_in_place():
    """300 steps (a 256-step captured chunk plus the rest), v_out aliasing v_in."""
    kw = dict(nx=32, ny=16, dt=0.02, Re=40.0)
    cfg = ns2d.Config(**kw)
    q = inputs.wake_like_field(16, 32, seed=7)
    v = inputs.gaussian_field(16, 32, seed=8)
    st = nsstab.Stepper(per_set=2, **kw)
    t = _dev(v)
    st.apply_tangent(_dev(q), t, t, 300 * cfg.dt)
    ref = ns2d.apply_tangent(q, v, 300 * cfg.dt, cfg)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


def test_newton_base_flow_matches_the_oracle():
    kw = dict(nx=32, ny=16, dt=0.02, Re=20.0)
    cfg = ns2d.Config(**kw)
    st = nsstab.Stepper(**kw)
    q = torch.zeros(16, 32, dtype=torch.float64, device="cuda")
    rc, r, iters, mv = st.newton_krylov_fixedpoint(q, T=0.4, gmres_m=40, tol=1e-10, max_newton=20)
    assert rc == nsstab.OK and r <= 1e-10 and iters <= 10 and mv > 0
    got = q.cpu().numpy()
    assert ns2d.residual(got, cfg) <= 2e-10
    ref = newton.newton_baseflow(cfg, np.zeros((16, 32)), T=0.4, tol=1e-10, max_newton=20, m=40)
    assert ref.converged
    assert np.abs(got - ref.x).max() <= 1e-8 * np.abs(ref.x).max()
    assert abs(iters - ref.iters) <= 1          # the same iteration (exact tangent on both sides)


def test_frozen_and_tangent_jacobians_reach_the_same_base_flow():
    kw = dict(nx=32, ny=16, dt=0.02, Re=40.0)
    cfg = ns2d.Config(**kw)
    q0 = ns2d.step_nonlinear(np.zeros((16, 32)), 20, cfg)
    out = {}
    for jac in ("tangent", "frozen"):
        st = nsstab.Stepper(**kw)
        q = _dev(q0)
        rc, r, iters, mv = st.newton_krylov_fixedpoint(q, T=0.4, gmres_m=40, tol=1e-10, max_newton=30,
                                                       gmres_rtol=1e-8, jacobian=jac)
        assert rc == nsstab.OK and r <= 1e-10
        out[jac] = (q.cpu().numpy(), iters)
    assert np.abs(out["tangent"][0] - out["frozen"][0]).max() <= 1e-8 * np.abs(out["tangent"][0]).max()
    assert out["tangent"][1] <= out["frozen"][1]


def test_mixed_precision_newton_reaches_the_fp64_residual_target():
    """FP32 Jacobian products, FP64 nonlinear map and residual (inexact Newton)."""
    kw = dict(nx=64, ny=32, dt=0.02, Re=30.0)
    cfg = ns2d.Config(**kw)
    st = nsstab.Stepper(**kw)
    lin = nsstab.Stepper(precision=32, **kw)
    q = _dev(ns2d.step_nonlinear(np.zeros((32, 64)), 50, cfg))
    rc, r, iters, mv = st.newton_krylov_fixedpoint(q, T=0.4, gmres_m=50, tol=1e-10, max_newton=30, lin=lin)
    assert rc == nsstab.OK and r <= 1e-10
    got = q.cpu().numpy()
    assert ns2d.residual(got, cfg) <= 2e-10
    mirror = got[(-np.arange(32)) % 32, :]
    assert np.abs(got + mirror).max() <= 1e-8 * np.abs(got).max()


def test_newton_rejects_mismatched_steppers():
    st = nsstab.Stepper(nx=32, ny=16, dt=0.02)
    other = nsstab.Stepper(nx=64, ny=32, dt=0.02)
    q = torch.zeros(16, 32, dtype=torch.float64, device="cuda")
    with pytest.raises(nsstab.NsstabError):
        st.newton_krylov_fixedpoint(q, T=0.4, gmres_m=10, tol=1e-10, max_newton=2, lin=other)


def test_cylinder_wake_leading_mode_is_the_shedding_pair():
    """Newton base flows at Re 40 and 60 (128x64) and the leading eigenvalues
    of M about them: a complex pair at the shedding frequency (St = omega/2pi
    in [0.11, 0.16] for D = U = 1), whose growth rate rises with Re."""
    growth = []
    for re in (40.0, 60.0):
        st = nsstab.Stepper(nx=128, ny=64, dt=0.01, Re=re)
        q = torch.zeros(64, 128, dtype=torch.float64, device="cuda")
        st.sfd_baseflow(q, chi=0.1, Delta=0.5, tol=0.0, max_steps=300, check_every=300)
        rc, r, iters, mv = st.newton_krylov_fixedpoint(q, T=0.4, gmres_m=50, tol=1e-10, max_newton=30)
        assert rc == nsstab.OK and r <= 1e-10
        got = q.cpu().numpy()
        mirror = got[(-np.arange(64)) % 64, :]
        assert np.abs(got + mirror).max() <= 1e-8 * np.abs(got).max()   # symmetric steady wake
        e = st.arnoldi_eigs(q, _dev(inputs.gaussian_field(64, 128, seed=0)), m=64, nev=2, tol=1e-10, T=0.5,
                            max_restarts=40)
        assert e.n_conv == len(e.mu)
        lam = e.growth(0.5)[0]
        assert e.mu[0].imag != 0.0 and 0.11 <= abs(lam.imag) / (2 * np.pi) <= 0.16
        growth.append(lam.real)
    assert growth[1] > growth[0]
