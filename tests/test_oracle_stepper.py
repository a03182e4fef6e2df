"""Pins of the oracle time-stepper against what the mathematics fixes.

None of these tests re-derives a value through the oracle's own code path:
each compares the oracle with an independent route (a spatial stencil, a
closed form, a scalar recurrence, a symmetry, an exact identity of a
quadratic map).
"""
import numpy as np
import pytest

from oracle import ns2d
from paper_1804_03859_gb300 import inputs


def _lap5(f, cfg):
    """5-point Laplacian written as a spatial stencil (not the Fourier symbol)."""
    return ((np.roll(f, -1, -1) - 2 * f + np.roll(f, 1, -1)) / cfg.dx ** 2
            + (np.roll(f, -1, -2) - 2 * f + np.roll(f, 1, -2)) / cfg.dy ** 2)


def _free_cfg(**kw):
    """No cylinder, no sponge: the periodic box alone."""
    base = dict(cyl_D=0.0, sponge_sigma=0.0)
    base.update(kw)
    return ns2d.Config(**base)


@pytest.mark.parametrize("nx,ny", [(32, 16), (128, 64), (64, 64)])
def test_poisson_satisfies_5pt_stencil(nx, ny):
    cfg = ns2d.Config(nx=nx, ny=ny)
    w = inputs.gaussian_field(ny, nx, seed=1)
    psi = ns2d.streamfunction(w, cfg)
    r = _lap5(psi, cfg) + w
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(w) * max(1.0, 1 / cfg.dx ** 2)
    assert abs(psi.mean()) < 1e-14 * np.abs(psi).max()


def _tg_mode(cfg, a, b):
    X, Y = ns2d.coords(cfg)
    kx = 2 * np.pi * a / cfg.Lx
    ky = 2 * np.pi * b / cfg.Ly
    # eigenvalue of the 5-point stencil on sin(kx x) sin(ky y)
    lam = (2 * np.cos(kx * cfg.dx) - 2) / cfg.dx ** 2 + (2 * np.cos(ky * cfg.dy) - 2) / cfg.dy ** 2
    return X, Y, kx, ky, lam


@pytest.mark.parametrize("a,b", [(2, 1), (5, 3)])
def test_taylor_green_discrete_closed_form(a, b):
    """omega^n = g^n omega^0, g = (1 + nu dt lam/2)/(1 - nu dt lam/2): advection vanishes."""
    cfg = _free_cfg(nx=64, ny=32, Uinf=0.0, Re=20.0, dt=0.01)
    X, Y, kx, ky, lam = _tg_mode(cfg, a, b)
    psi0 = np.sin(kx * X) * np.sin(ky * Y)
    w0 = -_lap5(psi0, cfg)
    n = 25
    got = ns2d.step_nonlinear(w0, n, cfg)
    g = (1 + 0.5 * cfg.nu * cfg.dt * lam) / (1 - 0.5 * cfg.nu * cfg.dt * lam)
    ref = g ** n * w0
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_taylor_green_advected_scalar_recurrence():
    """Uniform advection of one mode reduces to a complex scalar AB2/CN recurrence."""
    cfg = _free_cfg(nx=64, ny=32, Uinf=1.0, Re=40.0, dt=0.02)
    a, b = 3, 2
    X, Y, kx, ky, lam = _tg_mode(cfg, a, b)
    sx = np.sin(kx * cfg.dx) / cfg.dx       # symbol of the centred x-difference / i
    q = -1j * cfg.Uinf * sx                   # advection symbol: N = q c
    A = 1 + 0.5 * cfg.nu * cfg.dt * lam
    B = 1 - 0.5 * cfg.nu * cfg.dt * lam
    c_prev, c = None, -1j                     # omega = Re[c e^{i kx x}] sin(ky y)
    n = 40
    for k in range(n):
        if k == 0:
            c_new = (A * c + cfg.dt * q * c) / B
        else:
            c_new = (A * c + cfg.dt * (1.5 * q * c - 0.5 * q * c_prev)) / B
        c_prev, c = c, c_new
    w0 = np.sin(kx * X) * np.sin(ky * Y)
    ref = np.real(c * np.exp(1j * kx * X)) * np.sin(ky * Y)
    got = ns2d.step_nonlinear(w0, n, cfg)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_taylor_green_continuous_second_order():
    """Decay matches exp(-(kx^2+ky^2) nu t) with O(dx^2, dt^2) error."""
    errs = []
    T = 1.0
    for nx in (32, 64, 128):
        cfg = _free_cfg(nx=nx, ny=nx // 2, Uinf=0.0, Re=5.0, dt=0.05 * 32 / nx)
        X, Y, kx, ky, _ = _tg_mode(cfg, 2, 1)
        psi0 = np.sin(kx * X) * np.sin(ky * Y)
        w0 = (kx ** 2 + ky ** 2) * psi0           # continuous vorticity of the mode
        nsteps = ns2d.steps_per_period(T, cfg)
        got = ns2d.step_nonlinear(w0, nsteps, cfg)
        ref = np.exp(-(kx ** 2 + ky ** 2) * cfg.nu * T) * w0
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


@pytest.mark.parametrize("nx,ny,Lx,Ly", [(64, 32, 16.0, 8.0), (48, 64, 12.0, 4.0)])
def test_norm_h_is_the_continuous_l2_norm_of_trigonometric_fields(nx, ny, Lx, Ly):
    """On a periodic grid the rectangle rule integrates a trigonometric
    polynomial below the Nyquist degree exactly: the integral of
    sin^2(kx x) sin^2(ky y) over the box is Lx Ly / 4 and that of a constant c
    squared is c^2 Lx Ly.  A dropped or doubled cell area (dx dy) fails."""
    cfg = ns2d.Config(nx=nx, ny=ny, Lx=Lx, Ly=Ly)
    X, Y, kx, ky, _ = _tg_mode(cfg, 3, 2)
    f = np.sin(kx * X) * np.sin(ky * Y)
    assert abs(ns2d.norm_h(f, cfg) - np.sqrt(Lx * Ly) / 2) <= 1e-13 * np.sqrt(Lx * Ly)
    assert abs(ns2d.norm_h(np.full((ny, nx), -1.5), cfg) - 1.5 * np.sqrt(Lx * Ly)) <= 1e-13 * np.sqrt(Lx * Ly)
    both = np.stack([f, 2 * f])                     # leading axes are batch axes
    np.testing.assert_allclose(ns2d.norm_h(both, cfg), [np.sqrt(Lx * Ly) / 2, np.sqrt(Lx * Ly)], rtol=1e-13)


@pytest.mark.parametrize("a,b", [(2, 1), (4, 3)])
def test_residual_of_a_decaying_mode_is_its_discrete_decay(a, b):
    """Eq. 32's residual of a Taylor-Green mode in the free box: advection
    vanishes, one AB1/CN step multiplies the mode by g, so
    r = |g - 1| ||omega||_h / dt with ||omega||_h = |lam| sqrt(Lx Ly) / 2."""
    cfg = _free_cfg(nx=64, ny=32, Uinf=0.0, Re=30.0, dt=0.02)
    X, Y, kx, ky, lam = _tg_mode(cfg, a, b)
    w0 = -_lap5(np.sin(kx * X) * np.sin(ky * Y), cfg)
    g = (1 + 0.5 * cfg.nu * cfg.dt * lam) / (1 - 0.5 * cfg.nu * cfg.dt * lam)
    ref = abs(g - 1) * abs(lam) * np.sqrt(cfg.Lx * cfg.Ly) / 2 / cfg.dt
    assert abs(ns2d.residual(w0, cfg) - ref) <= 1e-10 * ref


def test_tangent_is_exact_derivative_of_quadratic_step():
    """G is quadratic in omega, so the central difference equals J v up to rounding."""
    cfg = ns2d.Config(nx=64, ny=32, dt=0.02)
    q = inputs.wake_like_field(32, 64, seed=3)
    v = inputs.gaussian_field(32, 64, seed=4)
    base = ns2d.Base.from_omega(q, cfg)
    jv, _ = ns2d.step(v, None, cfg, first=True, base=base)
    for eps in (1e-2, 1e-3):
        gp, _ = ns2d.step(q + eps * v, None, cfg, first=True)
        gm, _ = ns2d.step(q - eps * v, None, cfg, first=True)
        fd = (gp - gm) / (2 * eps)
        assert np.linalg.norm(fd - jv) <= 1e-9 * np.linalg.norm(jv)
    # and the forward difference is only first-order accurate (the map is not linear)
    gp, _ = ns2d.step(q + 1e-2 * v, None, cfg, first=True)
    g0, _ = ns2d.step(q, None, cfg, first=True)
    assert np.linalg.norm((gp - g0) / 1e-2 - jv) > 1e-6 * np.linalg.norm(jv)


def test_co_integrated_tangent_is_the_derivative_of_phi_T():
    """apply_tangent against central differences of the oracle's own
    nonlinear map over 10 steps: the error falls like eps^2, and the
    linearisation frozen at q (a different operator away from a fixed point)
    is far outside that error."""
    cfg = ns2d.Config(nx=64, ny=32, dt=0.02, Re=50.0)
    q = inputs.wake_like_field(32, 64, seed=5)
    v = inputs.smooth_field(32, 64, seed=6)
    T = 10 * cfg.dt
    jv = ns2d.apply_tangent(q, v, T, cfg)
    errs = []
    for eps in (1e-2, 1e-3):
        fd = (ns2d.step_nonlinear(q + eps * v, 10, cfg) - ns2d.step_nonlinear(q - eps * v, 10, cfg)) / (2 * eps)
        errs.append(np.linalg.norm(fd - jv) / np.linalg.norm(jv))
    assert errs[1] <= 1e-6 and 50 < errs[0] / errs[1] < 150, errs
    frozen = ns2d.apply_expTL(ns2d.Base.from_omega(q, cfg), v, T, cfg)
    assert np.linalg.norm(frozen - jv) / np.linalg.norm(jv) > 1e3 * errs[1]
    # one step: the tangent is the single linearised step about q
    one = ns2d.apply_tangent(q, v, cfg.dt, cfg)
    assert np.allclose(one, ns2d.step(v, None, cfg, first=True, base=ns2d.Base.from_omega(q, cfg))[0],
                       rtol=0, atol=1e-14 * np.abs(one).max())


def test_mean_free_and_mirror_symmetric_wake():
    """Impulsive start past a cylinder on the box's mid-line: the vorticity stays
    mean-free and antisymmetric, omega(x, Ly - y) = -omega(x, y)."""
    cfg = ns2d.Config(nx=64, ny=32, dt=0.02)
    w = ns2d.step_nonlinear(np.zeros((32, 64)), 100, cfg)
    assert np.abs(w).max() > 0.1
    assert abs(w.mean()) <= 1e-14 * np.abs(w).max()
    mirror = w[(-np.arange(32)) % 32, :]
    assert np.abs(w + mirror).max() <= 1e-11 * np.abs(w).max()


def test_penalisation_stops_flow_inside_cylinder():
    cfg = ns2d.Config(nx=128, ny=64, dt=0.01)
    w = ns2d.step_nonlinear(np.zeros((64, 128)), 200, cfg)
    u, v = ns2d.velocity(w, cfg)
    chi = ns2d.cylinder_mask(cfg)
    inside = chi >= 1.0
    assert inside.sum() > 10
    assert np.abs(u[inside]).max() < 0.2 and np.abs(v[inside]).max() < 0.2
    far = ns2d.coords(cfg)[0] < 1.0          # upstream, away from the body
    assert np.abs(u[far] - 1.0).max() < 0.2


def test_sponge_damps_perturbations_in_the_fringe():
    """With the base at rest in the free stream, a perturbation inside the fringe
    decays faster than one of the same shape outside it."""
    cfg = ns2d.Config(nx=128, ny=64, dt=0.01, cyl_D=0.0)
    base = ns2d.Base.from_omega(np.zeros((64, 128)), cfg)
    X, Y = ns2d.coords(cfg)

    def blob(xc):
        return np.exp(-((X - xc) ** 2 + (Y - 4.0) ** 2) / 0.3)

    def ratio(c):
        out_in = ns2d.step_linear(blob(15.2) - blob(15.2).mean(), 20, base, c)
        out_out = ns2d.step_linear(blob(8.0) - blob(8.0).mean(), 20, base, c)
        return np.linalg.norm(out_in) / np.linalg.norm(out_out)

    assert ratio(cfg) < 0.75
    cfg.sponge_sigma = 0.0
    assert ratio(cfg) > 0.95


def test_masks_shapes_and_ranges():
    cfg = ns2d.Config()
    chi = ns2d.cylinder_mask(cfg)
    sig = ns2d.sponge(cfg)
    assert chi.min() == 0.0 and chi.max() == 1.0
    assert np.all(sig >= 0.0) and sig.max() <= cfg.sponge_sigma
    X, _ = ns2d.coords(cfg)
    assert np.all(sig[X < 0.9 * cfg.Lx] == 0.0)
    # area of the smoothed disc ~ pi R^2
    area = chi.sum() * cfg.dx * cfg.dy
    assert abs(area - np.pi * 0.25) < 0.05
