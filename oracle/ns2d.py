"""Oracle: 2D incompressible Navier-Stokes time-stepper in vorticity-
streamfunction form (TEST INFRASTRUCTURE ONLY, see ``oracle/__init__``).

What the paper fixes
--------------------
Sec. 3 uses a time-stepper as a black box: it marches the nonlinear equations
(Eq. 28) to give the discrete map G of Eq. 2 / Eq. 41, and marches the
equations linearised about a base flow (Eq. 29, written dx/dt = A x in Eq. 30)
over a sampling period T to give the propagator M = exp(TA) of Eq. 42 / Eq. 55.
The paper does not describe the discretisation of its own solver, so the
scheme below is the one the workload specifies: doubly periodic box, second-
order centred finite differences, FFT solution of the 5-point Poisson problem,
Adams-Bashforth 2 for advection with Crank-Nicolson diffusion, a Brinkman-
penalised cylinder and a fringe sponge.  Each reading of an open point is
stated where it is made.

Grid: nx x ny vertices x_i = i dx, y_j = j dy (dx = Lx/nx, dy = Ly/ny), arrays
indexed ``[..., j, i]`` (x fastest), leading axes are batch axes.

Step (one call of ``step``), with nu = 1/Re:
  a1  psi = streamfunction(omega):  5-point Laplacian of psi = -omega, solved in
      Fourier space with the stencil's own symbol lam_h; the mean is zero.
  a2  N = -(u D_x omega + v D_y omega), u = Uinf + D_y psi, v = -D_x psi
      (linearised: N' = -(U_b D_x w + V_b D_y w + u' D_x Om_b + v' D_y Om_b)).
  a3  Crank-Nicolson / AB2 in Fourier space:
        (1 - nu dt lam_h/2) w* = (1 + nu dt lam_h/2) w^ + dt (3/2 N^n - 1/2 N^{n-1})
      (first step of every run: dt N^n), mean mode set to zero, psi* = -w*/lam_h.
  a4  implicit velocity-space Brinkman + sponge split:
        s = dt (chi/eta + sigma),
        du = (dt sigma Uinf - s u*)/(1+s), dv = -s v*/(1+s)   (linear: no dt sigma Uinf)
        omega^{n+1} = omega* + D_x dv - D_y du.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Config:
    """Physical and numerical parameters; defaults are the 128x64 cylinder case."""

    nx: int = 128
    ny: int = 64
    Lx: float = 16.0
    Ly: float = 8.0
    dt: float = 0.01
    Re: float = 50.0
    Uinf: float = 1.0
    cyl_x: float = 4.0
    cyl_y: float = 4.0
    cyl_D: float = 1.0          # 0 disables the cylinder
    eta: float = 1e-3           # Brinkman permeability
    mask_cells: float = 2.0     # width of the smoothed mask edge, in x-cells
    sponge_frac: float = 0.1    # fringe covers the last fraction of x
    sponge_sigma: float = 10.0  # peak fringe strength; 0 disables the sponge

    @property
    def dx(self) -> float:
        return self.Lx / self.nx

    @property
    def dy(self) -> float:
        return self.Ly / self.ny

    @property
    def nu(self) -> float:
        return 1.0 / self.Re

    @property
    def n(self) -> int:
        return self.nx * self.ny


# ----------------------------------------------------------------- geometry

def coords(cfg: Config):
    """Vertex coordinates X[j, i] = i dx, Y[j, i] = j dy."""
    x = np.arange(cfg.nx, dtype=np.float64) * cfg.dx
    y = np.arange(cfg.ny, dtype=np.float64) * cfg.dy
    return np.meshgrid(x, y)


def cylinder_mask(cfg: Config) -> np.ndarray:
    """Brinkman mask chi in [0, 1] of a cylinder of diameter D.

    Reading of "mask smoothed over 2 cells": chi = 1 for r <= R - w,
    0 for r >= R + w and (1 - sin(pi (r - R) / (2 w)))/2 in between, with
    R = D/2, w = mask_cells dx / 2 and r the periodic (minimum-image) distance.
    """
    if cfg.cyl_D <= 0.0:
        return np.zeros((cfg.ny, cfg.nx))
    X, Y = coords(cfg)
    ddx = np.mod(X - cfg.cyl_x + 0.5 * cfg.Lx, cfg.Lx) - 0.5 * cfg.Lx
    ddy = np.mod(Y - cfg.cyl_y + 0.5 * cfg.Ly, cfg.Ly) - 0.5 * cfg.Ly
    r = np.sqrt(ddx * ddx + ddy * ddy)
    R = 0.5 * cfg.cyl_D
    w = 0.5 * cfg.mask_cells * cfg.dx
    chi = 0.5 * (1.0 - np.sin(np.pi * (r - R) / (2.0 * w)))
    chi = np.where(r <= R - w, 1.0, chi)
    chi = np.where(r >= R + w, 0.0, chi)
    return chi


def sponge(cfg: Config) -> np.ndarray:
    """Fringe strength sigma(x): sigma_max sin^2(pi (x - xs)/(Lx - xs)) on x >= xs.

    Reading of "fringe sponge over the last 10% of x": xs = (1 - frac) Lx, a
    sin^2 ramp that is zero at both ends of the fringe.
    """
    if cfg.sponge_sigma <= 0.0 or cfg.sponge_frac <= 0.0:
        return np.zeros((cfg.ny, cfg.nx))
    X, _ = coords(cfg)
    xs = (1.0 - cfg.sponge_frac) * cfg.Lx
    ramp = np.sin(np.pi * (X - xs) / (cfg.sponge_frac * cfg.Lx)) ** 2
    return np.where(X >= xs, cfg.sponge_sigma * ramp, 0.0)


# ------------------------------------------------------ discrete operators

def ddx(f: np.ndarray, cfg: Config) -> np.ndarray:
    """Centred difference (f[i+1] - f[i-1]) / (2 dx), periodic."""
    return (np.roll(f, -1, axis=-1) - np.roll(f, 1, axis=-1)) / (2.0 * cfg.dx)


def ddy(f: np.ndarray, cfg: Config) -> np.ndarray:
    """Centred difference (f[j+1] - f[j-1]) / (2 dy), periodic."""
    return (np.roll(f, -1, axis=-2) - np.roll(f, 1, axis=-2)) / (2.0 * cfg.dy)


def laplacian_symbol(cfg: Config) -> np.ndarray:
    """Eigenvalues lam_h[ky, kx] of the periodic 5-point Laplacian on FFT modes."""
    kx = np.arange(cfg.nx, dtype=np.float64)
    ky = np.arange(cfg.ny, dtype=np.float64)
    lx = -(4.0 / cfg.dx ** 2) * np.sin(np.pi * kx / cfg.nx) ** 2
    ly = -(4.0 / cfg.dy ** 2) * np.sin(np.pi * ky / cfg.ny) ** 2
    return ly[:, None] + lx[None, :]


def _fft2(f):
    return np.fft.fft2(f, axes=(-2, -1))


def _ifft2_real(fh):
    return np.fft.ifft2(fh, axes=(-2, -1)).real


def _inverse_laplacian(fh: np.ndarray, cfg: Config) -> np.ndarray:
    """Return -fh / lam_h with the (0, 0) mode set to zero."""
    lam = laplacian_symbol(cfg).copy()
    lam[0, 0] = 1.0
    out = -fh / lam
    out[..., 0, 0] = 0.0
    return out


def streamfunction(omega: np.ndarray, cfg: Config) -> np.ndarray:
    """Step a1: psi with 5-point Laplacian(psi) = -omega, zero mean."""
    return _ifft2_real(_inverse_laplacian(_fft2(omega), cfg))


@dataclasses.dataclass
class Base:
    """Frozen base flow (Omega_b, Psi_b) about which Eq. 29 is linearised."""

    omega: np.ndarray
    psi: np.ndarray

    @classmethod
    def from_omega(cls, omega_b: np.ndarray, cfg: Config) -> "Base":
        return cls(omega=np.asarray(omega_b, dtype=np.float64),
                   psi=streamfunction(omega_b, cfg))


def advection_nonlinear(omega, psi, cfg: Config):
    """Step a2: N = -(u D_x omega + v D_y omega), u = Uinf + D_y psi, v = -D_x psi."""
    u = cfg.Uinf + ddy(psi, cfg)
    v = -ddx(psi, cfg)
    return -(u * ddx(omega, cfg) + v * ddy(omega, cfg))


def advection_linear(w, p, base: Base, cfg: Config):
    """Step a2, linearised about ``base`` (the advection terms of Eq. 29)."""
    Ub = cfg.Uinf + ddy(base.psi, cfg)
    Vb = -ddx(base.psi, cfg)
    u = ddy(p, cfg)
    v = -ddx(p, cfg)
    return -(Ub * ddx(w, cfg) + Vb * ddy(w, cfg)
             + u * ddx(base.omega, cfg) + v * ddy(base.omega, cfg))


def cn_ab2_update(omega_hat, N_hat, N_hat_prev, cfg: Config, first: bool):
    """Step a3: Crank-Nicolson diffusion, AB2 (AB1 on the first step) advection.

    Returns (omega_hat_star, psi_hat_star), both with the mean mode zeroed.
    """
    lam = laplacian_symbol(cfg)
    a = 1.0 + 0.5 * cfg.nu * cfg.dt * lam
    b = 1.0 - 0.5 * cfg.nu * cfg.dt * lam
    if first:
        R = N_hat
    else:
        R = 1.5 * N_hat - 0.5 * N_hat_prev
    wh = (a * omega_hat + cfg.dt * R) / b
    wh[..., 0, 0] = 0.0
    return wh, _inverse_laplacian(wh, cfg)


def penalize(omega_star, psi_star, cfg: Config, linear: bool):
    """Step a4: implicit Brinkman + fringe split in velocity space, then curl.

    Solves u^{n+1} = u* - dt (chi/eta) u^{n+1} - dt sigma (u^{n+1} - Uinf)
    (and the same for v with target 0) for the velocity correction and adds
    its discrete curl D_x dv - D_y du to the vorticity.  The linearised form
    has no target velocity.
    """
    chi = cylinder_mask(cfg)
    sig = sponge(cfg)
    s = cfg.dt * (chi / cfg.eta + sig)
    u = ddy(psi_star, cfg)
    if not linear:
        u = cfg.Uinf + u
    v = -ddx(psi_star, cfg)
    if linear:
        du = -s * u / (1.0 + s)
    else:
        du = (cfg.dt * sig * cfg.Uinf - s * u) / (1.0 + s)
    dv = -s * v / (1.0 + s)
    return omega_star + ddx(dv, cfg) - ddy(du, cfg)


def step(omega, N_hat_prev, cfg: Config, first: bool, base: Base | None = None):
    """One time step a1-a4.  ``base`` given => linearised step.

    Returns (omega_new, N_hat) where N_hat is this step's advection term in
    Fourier space (the AB2 history for the next step).
    """
    psi = streamfunction(omega, cfg)
    if base is None:
        N = advection_nonlinear(omega, psi, cfg)
    else:
        N = advection_linear(omega, psi, base, cfg)
    N_hat = _fft2(N)
    wh, ph = cn_ab2_update(_fft2(omega), N_hat, N_hat_prev, cfg, first)
    omega_new = penalize(_ifft2_real(wh), _ifft2_real(ph), cfg, linear=base is not None)
    return omega_new, N_hat


def step_nonlinear(omega0, nsteps: int, cfg: Config):
    """March the nonlinear equations nsteps steps (AB1 start): G^nsteps(omega0)."""
    omega = np.array(omega0, dtype=np.float64, copy=True)
    Nh = None
    for k in range(nsteps):
        omega, Nh = step(omega, Nh, cfg, first=(k == 0))
    return omega


def step_linear(v0, nsteps: int, base: Base, cfg: Config):
    """March the linearised equations nsteps steps about ``base`` (AB1 start)."""
    v = np.array(v0, dtype=np.float64, copy=True)
    Nh = None
    for k in range(nsteps):
        v, Nh = step(v, Nh, cfg, first=(k == 0), base=base)
    return v


def apply_tangent(q, v, T: float, cfg: Config):
    """Exact discrete tangent of the nonlinear map Phi_T (T/dt steps, AB1
    start) at q, applied to v: dPhi_T(q)/dq v.  The perturbation is advanced
    together with the trajectory (co-integration): step n linearises about
    the trajectory point q_n, and its AB2 history term is the linearised
    advection of step n-1 about q_{n-1}, which is the derivative of the
    two-step scheme itself.  The Newton-Krylov Jacobian of Sec. 3.1.2
    (Eq. 43) is I - apply_tangent."""
    nsteps = steps_per_period(T, cfg)
    w = np.array(q, dtype=np.float64, copy=True)
    dv = np.array(v, dtype=np.float64, copy=True)
    Nw = Nv = None
    for k in range(nsteps):
        base = Base.from_omega(w, cfg)
        dv, Nv = step(dv, Nv, cfg, first=(k == 0), base=base)
        w, Nw = step(w, Nw, cfg, first=(k == 0))
    return dv


def steps_per_period(T: float, cfg: Config) -> int:
    ns = T / cfg.dt
    k = int(round(ns))
    if k < 1 or abs(ns - k) > 1e-9 * max(1.0, ns):
        raise ValueError(f"T={T} is not a whole number of steps dt={cfg.dt}")
    return k


def apply_expTL(base: Base, v, T: float, cfg: Config):
    """Matrix-free propagator M v = exp(T A) v of Eq. 42 / Eq. 55.

    Every call starts from AB1 so that M is a fixed linear map of v alone.
    """
    return step_linear(v, steps_per_period(T, cfg), base, cfg)


def norm_h(f, cfg: Config):
    """Grid 2-norm sqrt(sum f^2 dx dy) over the last two axes."""
    return np.sqrt(np.sum(f * f, axis=(-2, -1)) * cfg.dx * cfg.dy)


def residual(q, cfg: Config) -> float:
    """Base-flow residual r(q) = ||G_1(q) - q||_h / dt, G_1 one AB1 step (Eq. 32)."""
    g, _ = step(np.asarray(q, dtype=np.float64), None, cfg, first=True)
    return float(norm_h(g - q, cfg) / cfg.dt)


def velocity(omega, cfg: Config):
    """Velocity (u, v) = (Uinf + D_y psi, -D_x psi) of a vorticity field."""
    psi = streamfunction(omega, cfg)
    return cfg.Uinf + ddy(psi, cfg), -ddx(psi, cfg)


def semidiscrete_linear_rhs(w, base: Base, cfg: Config):
    """Continuous-time linear operator A w of Eq. 30 for this discretisation.

    A w = N'(w) + nu lap_h w + curl(f), f = -(chi/eta + sigma) (u', v'),
    with the mean mode removed (the stepper zeroes it every step).  The
    stepper's M = exp(T A) + O(dt) (the penalisation split is first order).
    """
    psi = streamfunction(w, cfg)
    N = advection_linear(w, psi, base, cfg)
    lam = laplacian_symbol(cfg)
    diff = _ifft2_real(lam * _fft2(w))
    k = cylinder_mask(cfg) / cfg.eta + sponge(cfg)
    fu = -k * ddy(psi, cfg)
    fv = k * ddx(psi, cfg)
    out = N + cfg.nu * diff + ddx(fv, cfg) - ddy(fu, cfg)
    return out - out.mean(axis=(-2, -1), keepdims=True)


def mean_free(f):
    return f - np.mean(f, axis=(-2, -1), keepdims=True)
