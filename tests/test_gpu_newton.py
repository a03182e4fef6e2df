"""GPU Newton-Krylov base flow (Sec. 3.1.2, Eq. 43) against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import newton, ns2d  # noqa: E402
from paper_1804_03859_gb300 import inputs, nsstab  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


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
