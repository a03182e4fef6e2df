"""GPU parity of the FP32 step with fused row passes (four kernels a step:
column Poisson pass, fused right-hand-side row pass, column update, fused
penalisation row pass).  Same discrete operator as the six-kernel step, so
it is held to the FP32 bar against the FP64 oracle (1e-6 per step) and
checked against the six-kernel FP32 stepper, on grids and strip heights
that exercise one strip per unit and several side by side (G = 2048/nx),
the periodic wrap of the ring rows, batches with several parameter sets,
inactive members, selective frequency damping and graph-replayed runs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, krylov, ns2d, sfd  # noqa: E402
from paper_1804_03859_gb300 import inputs, nsstab  # noqa: E402

pytestmark = pytest.mark.gpu

TOL32 = 1e-6   # per step, as for the six-kernel FP32 stepper


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _cfg(nx, ny, **kw):
    c = dict(nx=nx, ny=ny, dt=0.01 * 128 / nx)
    c.update(kw)
    return c


CASES = [(64, 32, 2), (128, 64, 4), (256, 128, 16), (512, 256, 8), (1024, 64, 2), (2048, 1024, 16)]


@pytest.mark.parametrize("nx,ny,R", CASES)
def test_fused_nonlinear_and_linear_steps_match_the_oracle(nx, ny, R):
    kw = _cfg(nx, ny)
    cfg = ns2d.Config(**kw)
    st = nsstab.Stepper(precision=32, **kw)
    st.stepper_set_fused_rows(R)
    assert st.stepper_get_fused_rows() == R
    w0 = inputs.wake_like_field(ny, nx, seed=1) + 0.3 * inputs.smooth_field(ny, nx, seed=2, kmax=5)
    nst = 3
    t = _dev(w0)
    st.step_nonlinear(t, nst)
    assert _rel(_host(t), ns2d.step_nonlinear(w0, nst, cfg)) <= nst * TOL32
    base = inputs.wake_like_field(ny, nx, seed=3)
    v = inputs.gaussian_field(ny, nx, seed=4)
    out = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
    st.apply_expTL(_dev(base), _dev(v), out, nst * cfg.dt)
    ref = ns2d.apply_expTL(ns2d.Base.from_omega(base, cfg), v, nst * cfg.dt, cfg)
    assert _rel(_host(out), ref) <= nst * TOL32


@pytest.mark.parametrize("nx,ny,R", [(128, 64, 2), (512, 256, 16)])
def test_fused_and_six_kernel_fp32_steps_agree_over_a_graph_replayed_run(nx, ny, R):
    """300 linearised steps (a 256-step graph chunk plus a 44-step one): the
    fused and the six-kernel FP32 steppers differ by FP32 rounding only."""
    kw = _cfg(nx, ny)
    base = _dev(inputs.wake_like_field(ny, nx, seed=5))
    v = _dev(inputs.gaussian_field(ny, nx, seed=6))
    outs = []
    for fused in (0, R):
        st = nsstab.Stepper(precision=32, **kw)
        st.stepper_set_fused_rows(fused)
        o = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
        st.apply_expTL(base, v, o, 300 * kw["dt"])
        outs.append(_host(o))
    assert _rel(outs[1], outs[0]) <= 300 * TOL32
    # replaying the captured graphs gives bit-identical results
    st = nsstab.Stepper(precision=32, **kw)
    st.stepper_set_fused_rows(R)
    a = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    st.apply_expTL(base, v, a, 300 * kw["dt"])
    st.apply_expTL(base, v, b, 300 * kw["dt"])
    assert torch.equal(a, b)


def test_fused_batch_of_sets_and_members_matches_the_oracle_per_member():
    """Three Reynolds numbers x two members each (each set its own base
    flow): every member against the oracle's propagator for its set."""
    nx, ny, R = 128, 64, 4
    Res = [40.0, 60.0, 90.0]
    kw = _cfg(nx, ny)
    st = nsstab.Stepper(precision=32, Re=Res, per_set=2, **kw)
    st.stepper_set_fused_rows(R)
    bases = np.stack([inputs.wake_like_field(ny, nx, seed=20 + k) for k in range(3)])
    v = np.stack([inputs.gaussian_field(ny, nx, seed=30 + m) for m in range(6)])
    out = torch.empty(6, ny, nx, dtype=torch.float64, device="cuda")
    nst = 4
    st.apply_expTL(_dev(bases), _dev(v), out, nst * kw["dt"])
    got = _host(out)
    for m in range(6):
        cfg = ns2d.Config(Re=Res[m // 2], **kw)
        ref = ns2d.apply_expTL(ns2d.Base.from_omega(bases[m // 2], cfg), v[m], nst * kw["dt"], cfg)
        assert _rel(got[m], ref) <= nst * TOL32, m


def test_fused_rows_sfd_trajectory_tracks_the_oracle():
    kw = _cfg(64, 32, dt=0.02, Re=40.0)
    cfg = ns2d.Config(**kw)
    w0 = inputs.wake_like_field(32, 64, seed=11)
    st = nsstab.Stepper(precision=32, **kw)
    st.stepper_set_fused_rows(4)
    t = _dev(w0)
    rc, r, steps = st.sfd_baseflow(t, chi=0.5, Delta=1.0, tol=0.0, max_steps=120, check_every=40)
    assert rc == nsstab.NOT_CONVERGED and steps == 120
    X, rr, k, ok = sfd.sfd_baseflow(cfg, w0, 0.5, 1.0, tol=0.0, max_steps=120, check_every=40)
    assert _rel(_host(t), X) <= 120 * TOL32
    assert abs(r - rr) <= 1e-3 * rr


def test_fused_rows_batched_krylov_with_members_leaving():
    """Batched Krylov-Schur (members finish at different rounds and stop
    being stepped) through the fused passes: every member's leading
    eigenvalues against the dense eigendecomposition of its assembled M."""
    kw = dict(nx=64, ny=32, dt=0.02)
    T = 1.0
    Res = [45.0, 70.0]
    bases = np.stack([inputs.wake_like_field(32, 64, seed=7 + k) for k in range(2)])
    st = nsstab.Stepper(precision=32, Re=Res, **kw)
    st.stepper_set_fused_rows(2)
    v0 = np.stack([inputs.gaussian_field(32, 64, seed=50 + k) for k in range(2)])
    res = st.batch_arnoldi_eigs(_dev(bases), _dev(v0), m=48, nev=4, tol=1e-6, T=T, max_restarts=60)
    for k, r in enumerate(res):
        cfg = ns2d.Config(Re=Res[k], **kw)
        M = dense.assemble_M(ns2d.Base.from_omega(bases[k], cfg), T, cfg)
        mu = np.linalg.eigvals(M)
        mu = mu[krylov.leading_order(mu)][:6]
        assert r.n_conv == len(r.mu)
        for x in r.mu:
            assert np.min(np.abs(mu - x)) <= 1e-5 * abs(x)


def test_fused_rows_default_and_rejections():
    st = nsstab.Stepper(precision=32, **_cfg(256, 128))
    assert st.stepper_get_fused_rows() == 0      # off by default
    st.stepper_set_fused_rows(8)
    st.stepper_set_fused_rows(0)
    assert st.stepper_get_fused_rows() == 0
    for prec, nx, ny, R in [(64, 128, 64, 4), (48, 128, 64, 4), (32, 32, 16, 2), (32, 128, 64, 3),
                            (32, 128, 64, 128), (32, 4096, 64, 2)]:
        st = nsstab.Stepper(precision=prec, **_cfg(nx, ny))
        with pytest.raises(nsstab.NsstabError):
            st.stepper_set_fused_rows(R)
        assert st.stepper_get_fused_rows() == 0
