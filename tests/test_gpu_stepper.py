"""GPU parity of the time-stepper (steps a1-a5) against the FP64 oracle.

Bar: relative L2 error <= 1e-12 per FP64 step (1e-6 per FP32 step), on
seeded synthetic fields, at sizes from a single tile up to the largest
workload grids, every call going through the C ABI.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns2d, sfd  # noqa: E402
from paper_1804_03859_gb300 import inputs, nsstab  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _tol32(nx, ny):
    """FP32 bound per step.  The FP32 stepper forms the velocities from the
    spectrum of psi (the centred-difference symbols), so no difference of a
    rounded psi is taken and the error stays a few FP32 roundings (measured
    1.2e-7 ... 4.2e-7 from 128x64 to 2048x1024) instead of growing like
    eps32 / (dx dy)."""
    return 1e-6


def _cfg(nx, ny, **kw):
    c = dict(nx=nx, ny=ny, dt=0.01 * 128 / nx)
    c.update(kw)
    return c


GRIDS = [(8, 8), (16, 8), (32, 16), (128, 64), (64, 256), (256, 32), (512, 256)]


@pytest.mark.parametrize("nx,ny", GRIDS)
def test_poisson_parity(nx, ny):
    kw = _cfg(nx, ny)
    st = nsstab.Stepper(**kw)
    w = inputs.gaussian_field(ny, nx, seed=nx + ny)
    psi = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    st.stepper_poisson(_dev(w), psi)
    ref = ns2d.streamfunction(w, ns2d.Config(**kw))
    assert _rel(_host(psi), ref) <= 1e-13


@pytest.mark.parametrize("nx,ny", GRIDS)
def test_fp32_poisson_parity(nx, ny):
    """The FP32 stepper carries velocities in its step; its Poisson entry
    forms psi through the row-pair variant of the inverse pass (with the
    block shrunk where the velocity plan is wider than ny/2 pairs)."""
    kw = _cfg(nx, ny)
    st = nsstab.Stepper(precision=32, **kw)
    w = inputs.gaussian_field(ny, nx, seed=nx + ny)
    psi = torch.zeros(ny, nx, dtype=torch.float64, device="cuda")
    st.stepper_poisson(_dev(w), psi)
    ref = ns2d.streamfunction(w, ns2d.Config(**kw))
    assert _rel(_host(psi), ref) <= 1e-6


def test_fp32_sfd_trajectory_tracks_the_oracle():
    """Selective frequency damping through the FP32 penalisation pass (the
    velocity form of the SFD-forced step)."""
    kw = _cfg(64, 32, dt=0.02, Re=40.0)
    cfg = ns2d.Config(**kw)
    w0 = inputs.wake_like_field(32, 64, seed=11)
    st = nsstab.Stepper(precision=32, **kw)
    t = _dev(w0)
    rc, r, steps = st.sfd_baseflow(t, chi=0.5, Delta=1.0, tol=0.0, max_steps=120, check_every=40)
    assert rc == nsstab.NOT_CONVERGED and steps == 120
    X, rr, k, ok = sfd.sfd_baseflow(cfg, w0, 0.5, 1.0, tol=0.0, max_steps=120, check_every=40)
    assert _rel(_host(t), X) <= 120 * _tol32(64, 32)
    assert abs(r - rr) <= 1e-3 * rr


@pytest.mark.parametrize("nx,ny", GRIDS)
def test_one_nonlinear_step_parity(nx, ny):
    kw = _cfg(nx, ny)
    cfg = ns2d.Config(**kw)
    w0 = inputs.wake_like_field(ny, nx, seed=1) + 0.3 * inputs.smooth_field(ny, nx, seed=2, kmax=5)
    st = nsstab.Stepper(**kw)
    t = _dev(w0)
    st.step_nonlinear(t, 1)
    ref = ns2d.step_nonlinear(w0, 1, cfg)
    assert _rel(_host(t), ref) <= 1e-12


def test_many_nonlinear_steps_parity_and_invariants():
    kw = _cfg(128, 64)
    cfg = ns2d.Config(**kw)
    st = nsstab.Stepper(**kw)
    t = torch.zeros(64, 128, dtype=torch.float64, device="cuda")
    st.step_nonlinear(t, 60)
    got = _host(t)
    ref = ns2d.step_nonlinear(np.zeros((64, 128)), 60, cfg)
    assert _rel(got, ref) <= 60 * 1e-12
    assert abs(got.mean()) <= 1e-13 * np.abs(got).max()
    mirror = got[(-np.arange(64)) % 64, :]
    assert np.abs(got + mirror).max() <= 1e-10 * np.abs(got).max()


@pytest.mark.parametrize("nx,ny", [(32, 16), (128, 64), (256, 128)])
def test_linear_step_and_propagator_parity(nx, ny):
    kw = _cfg(nx, ny)
    cfg = ns2d.Config(**kw)
    base = inputs.wake_like_field(ny, nx, seed=3)
    v = inputs.gaussian_field(ny, nx, seed=4)
    st = nsstab.Stepper(**kw)
    out = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
    st.apply_expTL(_dev(base), _dev(v), out, cfg.dt)        # one step
    b = ns2d.Base.from_omega(base, cfg)
    ref1, _ = ns2d.step(v, None, cfg, first=True, base=b)
    assert _rel(_host(out), ref1) <= 1e-12
    T = 20 * cfg.dt
    st.apply_expTL(None, _dev(v), out, T)                   # the kept base
    refT = ns2d.apply_expTL(b, v, T, cfg)
    assert _rel(_host(out), refT) <= ns2d.steps_per_period(T, cfg) * 1e-12


def test_propagator_in_place_and_zero_steps():
    kw = _cfg(64, 32)
    st = nsstab.Stepper(**kw)
    base = _dev(inputs.wake_like_field(32, 64, seed=5))
    v = _dev(inputs.gaussian_field(32, 64, seed=6))
    other = torch.empty_like(v)
    st.apply_expTL(base, v, other, 0.2)
    inplace = v.clone()
    st.apply_expTL(None, inplace, inplace, 0.2)
    assert torch.equal(other, inplace)
    w = v.clone()
    st.step_nonlinear(w, 0)
    assert torch.equal(w, v)
    with pytest.raises(nsstab.NsstabError):
        st.apply_expTL(None, v, other, 0.2 + 0.5 * st.cfg.dt)


def test_propagator_is_linear():
    kw = _cfg(64, 32)
    st = nsstab.Stepper(**kw)
    st.stepper_set_base(_dev(inputs.wake_like_field(32, 64, seed=7)))
    a = inputs.gaussian_field(32, 64, seed=8)
    b = inputs.gaussian_field(32, 64, seed=9)
    outs = []
    for v in (a, b, 2.0 * a - 3.0 * b):
        o = torch.empty(32, 64, dtype=torch.float64, device="cuda")
        st.apply_expTL(None, _dev(v), o, 0.3)
        outs.append(_host(o))
    assert _rel(outs[2], 2.0 * outs[0] - 3.0 * outs[1]) <= 1e-12


def test_residual_parity():
    kw = _cfg(128, 64)
    cfg = ns2d.Config(**kw)
    q = inputs.wake_like_field(64, 128, seed=10)
    st = nsstab.Stepper(**kw)
    r = st.stepper_residual(_dev(q))
    assert abs(r - ns2d.residual(q, cfg)) <= 1e-12 * ns2d.residual(q, cfg)


def test_sfd_trajectory_parity():
    kw = _cfg(64, 32, dt=0.02, Re=40.0)
    cfg = ns2d.Config(**kw)
    w0 = inputs.wake_like_field(32, 64, seed=11)
    st = nsstab.Stepper(**kw)
    t = _dev(w0)
    rc, r, steps = st.sfd_baseflow(t, chi=0.5, Delta=1.0, tol=0.0, max_steps=120, check_every=40)
    assert rc == nsstab.NOT_CONVERGED and steps == 120
    X, rr, k, ok = sfd.sfd_baseflow(cfg, w0, 0.5, 1.0, tol=0.0, max_steps=120, check_every=40)
    assert _rel(_host(t), X) <= 120 * 1e-12
    assert abs(r - rr) <= 1e-9 * rr


def test_sfd_reaches_the_base_flow_residual_target():
    kw = _cfg(32, 16, dt=0.02, Re=20.0)
    cfg = ns2d.Config(**kw)
    st = nsstab.Stepper(**kw)
    t = torch.zeros(16, 32, dtype=torch.float64, device="cuda")
    rc, r, steps = st.sfd_baseflow(t, chi=0.5, Delta=1.0, tol=1e-10, max_steps=40000, check_every=200)
    assert rc == nsstab.OK and r <= 1e-10
    q = _host(t)
    assert ns2d.residual(q, cfg) <= 2e-10
    X, rr, k, ok = sfd.sfd_baseflow(cfg, np.zeros((16, 32)), 0.5, 1.0, tol=1e-10, max_steps=40000, check_every=200)
    assert ok and abs(k - steps) <= 200
    assert np.abs(q - X).max() <= 1e-8 * np.abs(X).max()


@pytest.mark.parametrize("nx,ny", [(128, 64), (512, 256)])
def test_fp32_stepper_tracks_the_fp64_oracle(nx, ny):
    kw = _cfg(nx, ny)
    cfg = ns2d.Config(**kw)
    w0 = inputs.wake_like_field(ny, nx, seed=12)
    st = nsstab.Stepper(precision=32, **kw)
    t = _dev(w0)
    st.step_nonlinear(t, 1)
    assert _rel(_host(t), ns2d.step_nonlinear(w0, 1, cfg)) <= _tol32(nx, ny)
    base = inputs.wake_like_field(ny, nx, seed=13)
    v = inputs.gaussian_field(ny, nx, seed=14)
    out = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
    st.apply_expTL(_dev(base), _dev(v), out, 5 * cfg.dt)
    ref = ns2d.apply_expTL(ns2d.Base.from_omega(base, cfg), v, 5 * cfg.dt, cfg)
    assert _rel(_host(out), ref) <= 5 * _tol32(nx, ny)


def test_fp32_smooth_perturbation_at_fine_grid():
    """A smooth perturbation on a fine grid is where a centred difference of
    a rounded psi cancels most (|psi| / (h |D psi|) is largest): one
    linearised FP32 step must still be within 1e-6 of the FP64 oracle."""
    nx, ny = 512, 256
    kw = _cfg(nx, ny)
    cfg = ns2d.Config(**kw)
    base = inputs.wake_like_field(ny, nx, seed=31)
    v = inputs.smooth_field(ny, nx, seed=32, kmax=6)
    st = nsstab.Stepper(precision=32, **kw)
    out = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
    st.apply_expTL(_dev(base), _dev(v), out, cfg.dt)
    ref = ns2d.apply_expTL(ns2d.Base.from_omega(base, cfg), v, cfg.dt, cfg)
    assert _rel(_host(out), ref) <= _tol32(nx, ny)
    psi = torch.empty_like(out)
    st.stepper_poisson(_dev(base), psi)
    assert _rel(_host(psi), ns2d.streamfunction(base, cfg)) <= _tol32(nx, ny)


@pytest.mark.parametrize("nx,ny,prec", [(2048, 1024, 64), (2048, 1024, 32), (4096, 2048, 64), (4096, 2048, 32)])
def test_full_size_single_step(nx, ny, prec):
    """Largest workload grids: one nonlinear and one linearised step."""
    kw = _cfg(nx, ny)
    cfg = ns2d.Config(**kw)
    w0 = inputs.wake_like_field(ny, nx, seed=15)
    st = nsstab.Stepper(precision=prec, **kw)
    t = _dev(w0)
    st.step_nonlinear(t, 1)
    tol = 1e-12 if prec == 64 else _tol32(nx, ny)
    assert _rel(_host(t), ns2d.step_nonlinear(w0, 1, cfg)) <= tol
    v = inputs.gaussian_field(ny, nx, seed=16)
    out = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
    st.apply_expTL(_dev(w0), _dev(v), out, cfg.dt)
    ref, _ = ns2d.step(v, None, cfg, first=True, base=ns2d.Base.from_omega(w0, cfg))
    assert _rel(_host(out), ref) <= tol


def test_every_launch_plan_gives_the_same_step():
    """Each kernel under every valid (elements per thread, sequences per block)
    plan reproduces the oracle step: the plans change the radix and the launch
    shape, never the method."""
    kw = _cfg(64, 32)
    cfg = ns2d.Config(**kw)
    w0 = inputs.wake_like_field(32, 64, seed=21)
    base = inputs.wake_like_field(32, 64, seed=22)
    v = inputs.gaussian_field(32, 64, seed=23)
    ref_nl = ns2d.step_nonlinear(w0, 3, cfg)
    ref_lin = ns2d.apply_expTL(ns2d.Base.from_omega(base, cfg), v, 3 * cfg.dt, cfg)
    st = nsstab.Stepper(**kw)
    defaults = st.plans()
    tried = 0
    for kid in range(6):
        for le in (1, 2, 3):
            for per in (1, 2, 4, 8):
                try:
                    st.stepper_set_plan(kid, le, per)
                except nsstab.NsstabError:
                    continue
                tried += 1
                t = _dev(w0)
                st.step_nonlinear(t, 3)
                assert _rel(_host(t), ref_nl) <= 3e-12, (kid, le, per)
                out = torch.empty(32, 64, dtype=torch.float64, device="cuda")
                st.apply_expTL(_dev(base), _dev(v), out, 3 * cfg.dt)
                assert _rel(_host(out), ref_lin) <= 3e-12, (kid, le, per)
        st.stepper_set_plan(kid, *defaults[nsstab.Stepper.KERNELS[kid]])
    assert tried >= 30
    with pytest.raises(nsstab.NsstabError):
        st.stepper_set_plan(0, 4, 1)


@pytest.mark.parametrize("nx,ny,prec", [(128, 64, 64), (512, 256, 64), (128, 64, 32), (512, 256, 32)])
def test_autotuned_plans_keep_parity(nx, ny, prec):
    kw = _cfg(nx, ny)
    cfg = ns2d.Config(**kw)
    st = nsstab.Stepper(precision=prec, **kw)
    chosen = st.stepper_autotune(reps=3)
    assert set(chosen) == set(nsstab.Stepper.KERNELS)
    assert st.plans() == chosen
    w0 = inputs.wake_like_field(ny, nx, seed=24)
    t = _dev(w0)
    st.step_nonlinear(t, 2)
    tol = 2e-12 if prec == 64 else 2 * _tol32(nx, ny)
    assert _rel(_host(t), ns2d.step_nonlinear(w0, 2, cfg)) <= tol


def test_long_runs_through_several_graph_chunks():
    """300 steps: one captured 256-step chunk plus a 44-step chunk."""
    kw = _cfg(64, 32, dt=0.02)
    cfg = ns2d.Config(**kw)
    st = nsstab.Stepper(**kw)
    t = torch.zeros(32, 64, dtype=torch.float64, device="cuda")
    st.step_nonlinear(t, 300)
    ref = ns2d.step_nonlinear(np.zeros((32, 64)), 300, cfg)
    assert _rel(_host(t), ref) <= 300 * 1e-12
    # replaying the cached graphs gives bit-identical results
    t2 = torch.zeros(32, 64, dtype=torch.float64, device="cuda")
    st.step_nonlinear(t2, 300)
    assert torch.equal(t, t2)


# ---------------------------------------------------------------- double-float

@pytest.mark.parametrize("nx,ny", [(16, 8), (128, 64), (64, 256), (512, 256), (2048, 1024)])
def test_double_float_stepper_within_1e12_per_step_up_to_512x256_then_scaled(nx, ny):
    """precision 48: FP32-pair arithmetic.  Held to the FP64 bar (1e-12 per
    step) up to the 512x256 workload grid; beyond it the bound grows with the
    grid density (2e-12 at 1024x512, 4e-12 at 2048x1024), because the unit
    roundoff (2^-48) is 32 times FP64's and the centred differences of psi
    lose ~eps/(dx dy) to cancellation (measured 1.4e-12 at 2048x1024).  So
    the double-float stepper is FP64-class only up to 512x256."""
    kw = _cfg(nx, ny)
    cfg = ns2d.Config(**kw)
    w0 = inputs.wake_like_field(ny, nx, seed=1) + 0.3 * inputs.smooth_field(ny, nx, seed=2, kmax=5)
    st = nsstab.Stepper(precision=48, **kw)
    t = _dev(w0)
    st.step_nonlinear(t, 1)
    tol = max(1e-12, 1e-12 * (nx / 512.0) * (ny / 256.0) / 4.0)
    assert _rel(_host(t), ns2d.step_nonlinear(w0, 1, cfg)) <= tol
    base = inputs.wake_like_field(ny, nx, seed=3)
    v = inputs.gaussian_field(ny, nx, seed=4)
    out = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
    nsteps = 20 if nx <= 512 else 2
    st.apply_expTL(_dev(base), _dev(v), out, nsteps * cfg.dt)
    ref = ns2d.apply_expTL(ns2d.Base.from_omega(base, cfg), v, nsteps * cfg.dt, cfg)
    assert _rel(_host(out), ref) <= nsteps * tol


def test_double_float_autotuned_plans_keep_parity():
    kw = _cfg(256, 128)
    cfg = ns2d.Config(**kw)
    st = nsstab.Stepper(precision=48, **kw)
    st.stepper_autotune(reps=3)
    w0 = inputs.wake_like_field(128, 256, seed=5)
    t = _dev(w0)
    st.step_nonlinear(t, 3)
    assert _rel(_host(t), ns2d.step_nonlinear(w0, 3, cfg)) <= 3e-12
