"""Failure detection without any GPU fault: non-finite data injected on the
host surfaces as NSSTAB_DIVERGED from the solvers, bad arguments as
NSSTAB_ERR_INVALID_ARG, and the stepper stays usable afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns2d  # noqa: E402
from paper_1804_03859_gb300 import inputs, nsstab  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _nan_field(ny, nx):
    f = inputs.wake_like_field(ny, nx, seed=1)
    f[ny // 2, nx // 3] = np.nan
    return f


def test_non_finite_state_is_reported_and_the_stepper_recovers():
    kw = dict(nx=64, ny=32, dt=0.02)
    cfg = ns2d.Config(**kw)
    st = nsstab.Stepper(**kw)
    rc, r, steps = st.sfd_baseflow(_dev(_nan_field(32, 64)), chi=0.5, Delta=1.0, tol=1e-10, max_steps=400,
                                   check_every=100)
    assert rc == nsstab.DIVERGED and not np.isfinite(r)
    r = st.stepper_residual(_dev(_nan_field(32, 64)))
    assert not np.isfinite(r)
    q = torch.zeros(32, 64, dtype=torch.float64, device="cuda")
    rc, r, it, mv = st.newton_krylov_fixedpoint(_dev(_nan_field(32, 64)), T=0.4, gmres_m=5, tol=1e-10, max_newton=3)
    assert rc == nsstab.DIVERGED
    # the same stepper still computes correct steps afterwards
    w0 = inputs.wake_like_field(32, 64, seed=2)
    t = _dev(w0)
    st.step_nonlinear(t, 2)
    ref = ns2d.step_nonlinear(w0, 2, cfg)
    assert np.linalg.norm(t.cpu().numpy() - ref) <= 2e-12 * np.linalg.norm(ref)


def test_non_finite_base_flow_stops_the_eigen_solver():
    st = nsstab.Stepper(nx=32, ny=16, dt=0.02)
    v0 = _dev(inputs.gaussian_field(16, 32, seed=3))
    res = st.arnoldi_eigs(_dev(_nan_field(16, 32)), v0, m=10, nev=2, tol=1e-8, T=0.2)
    assert res.status == nsstab.DIVERGED


def test_invalid_arguments_are_rejected_before_launch():
    st = nsstab.Stepper(nx=32, ny=16, dt=0.02)
    t = torch.zeros(16, 32, dtype=torch.float64, device="cuda")
    with pytest.raises(nsstab.NsstabError):
        st.sfd_baseflow(t, chi=0.5, Delta=0.0, tol=1e-10, max_steps=10)
    with pytest.raises(nsstab.NsstabError):
        st.step_nonlinear(t, -1)
    with pytest.raises(ValueError):
        st.step_nonlinear(torch.zeros(16, 33, dtype=torch.float64, device="cuda"), 1)
    with pytest.raises(ValueError):
        st.step_nonlinear(torch.zeros(16, 32, dtype=torch.float32, device="cuda"), 1)
