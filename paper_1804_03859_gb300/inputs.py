"""Seeded synthetic inputs shared by the tests, the smoke run and the bench.

This module holds no arithmetic of the method: it only draws random numbers
and evaluates closed-form fields on the grid.  Everything is float64, shaped
``[ny, nx]`` (x fastest), and reproducible from ``seed`` with numpy's
``default_rng``.
"""
from __future__ import annotations

import numpy as np


def gaussian_field(ny: int, nx: int, seed: int, unit_norm: bool = True) -> np.ndarray:
    """Seeded Gaussian vector, mean removed, optionally of unit Euclidean norm.

    This is the Arnoldi starting vector of the cylinder workloads.
    """
    f = np.random.default_rng(seed).standard_normal((ny, nx))
    f -= f.mean()
    if unit_norm:
        f /= np.linalg.norm(f)
    return f


def smooth_field(ny: int, nx: int, seed: int, Lx: float = 16.0, Ly: float = 8.0,
                 kmax: int = 4, amp: float = 1.0) -> np.ndarray:
    """Sum of random low-wavenumber periodic modes (|k| <= kmax), zero mean."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) * (Lx / nx)
    y = np.arange(ny) * (Ly / ny)
    X, Y = np.meshgrid(x, y)
    f = np.zeros((ny, nx))
    for a in range(0, kmax + 1):
        for b in range(-kmax, kmax + 1):
            if a == 0 and b <= 0:
                continue
            c, s = rng.standard_normal(2) / (1.0 + a * a + b * b)
            ph = 2 * np.pi * (a * X / Lx + b * Y / Ly)
            f += c * np.cos(ph) + s * np.sin(ph)
    f -= f.mean()
    return amp * f / np.abs(f).max()


def wake_like_field(ny: int, nx: int, seed: int, Lx: float = 16.0, Ly: float = 8.0,
                    cyl_x: float = 4.0, cyl_y: float = 4.0, noise: float = 0.05) -> np.ndarray:
    """A developed-wake-shaped vorticity field: two opposite-signed shear
    layers trailing the cylinder position, with a seeded perturbation.

    It stands in for a base flow where only the field's shape and scale
    matter (throughput runs and parity of the linearised stepper); it is not
    a steady state.
    """
    x = np.arange(nx) * (Lx / nx)
    y = np.arange(ny) * (Ly / ny)
    X, Y = np.meshgrid(x, y)
    downstream = np.clip((X - cyl_x) / 1.0, 0.0, 1.0) * np.exp(-np.clip(X - cyl_x, 0, None) / 6.0)
    layer = (np.exp(-((Y - cyl_y - 0.5) / 0.25) ** 2) - np.exp(-((Y - cyl_y + 0.5) / 0.25) ** 2))
    f = 2.0 * downstream * layer
    f += noise * smooth_field(ny, nx, seed, Lx, Ly, kmax=6)
    return f - f.mean()
