"""Seeded synthetic initial fields (rho', u', theta') shared by tests, benchmark and oracle runs.

This module only draws random numbers and samples smooth functions on the grid; it holds none of
the lattice Boltzmann arithmetic.  All fields are FP64 numpy arrays in the library layout:
rho[cells], u[D][cells], theta[cells], cell = x + nx * (y + ny * z).

Workloads follow the paper's test problem (Sec. 9): Gauss pulses in the density with zero
velocity and temperature perturbation on periodic grids, here with sizes, amplitudes and seeds
of the benchmark configurations, plus density plane waves for the 2D field.
"""
from __future__ import annotations

import numpy as np


def _coords(shape):
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.ravel().astype(np.float64), y.ravel().astype(np.float64), z.ravel().astype(np.float64)


def gaussian_pulse(shape, amplitude: float, width: float, center, periodic: bool = True) -> np.ndarray:
    """amplitude * exp(-|x - center|^2 / width^2) on the grid, with minimum-image distances on a
    periodic grid.  Same form as the paper's exp(-a |x - x0|^2) with a = 1 / width^2."""
    dims = [d for d in (list(shape) + [1, 1])[:3]]
    X = _coords(shape)
    r2 = np.zeros(X[0].shape)
    for a in range(3):
        if dims[a] == 1:
            continue
        d = X[a] - center[a]
        if periodic:
            d = (d + dims[a] / 2.0) % dims[a] - dims[a] / 2.0
        r2 += d * d
    return amplitude * np.exp(-r2 / (width * width))


def plane_wave(shape, amplitude: float, m, phase: float) -> np.ndarray:
    """amplitude * cos(2 pi (m_x x / nx + m_y y / ny + m_z z / nz) + phase) with integer m, so
    that the wave is periodic on the grid."""
    dims = (list(shape) + [1, 1])[:3]
    X = _coords(shape)
    arg = sum(2 * np.pi * m[a] * X[a] / dims[a] for a in range(3) if dims[a] > 1)
    return amplitude * np.cos(arg + phase)


def zero_rest(D: int, cells: int):
    return np.zeros((D, cells)), np.zeros(cells)


def config_1d(n: int = 1024, seed: int = 1):
    """1D: Gaussian pressure pulse, amplitude 1e-3, width 20 cells, centre ~ U[0, n)."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0, n)
    rho = gaussian_pulse((n, 1, 1), 1e-3, 20.0, (x0, 0, 0))
    u, th = zero_rest(1, n)
    return rho, u, th


def config_2d(n: int = 2048, seed: int = 2, n_waves: int = 8):
    """2D: Gaussian pulse (amplitude 1e-3, width 32 cells, centre ~ U) plus n_waves density plane
    waves of amplitude 1e-4 with random integer wave vectors whose wavelength n / |m| lies in
    [16, 256] cells (scaled with n / 2048 on smaller grids), random direction and phase."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, n, size=2)
    rho = gaussian_pulse((n, n, 1), 1e-3, 32.0, (c[0], c[1], 0))
    lo, hi = max(1.0, n / 256.0), max(1.0, n / 16.0)
    for _ in range(n_waves):
        while True:
            kmag = rng.uniform(lo, hi)
            ang = rng.uniform(0, 2 * np.pi)
            m = (int(round(kmag * np.cos(ang))), int(round(kmag * np.sin(ang))), 0)
            if m[0] != 0 or m[1] != 0:
                break
        rho += plane_wave((n, n, 1), 1e-4, m, rng.uniform(0, 2 * np.pi))
    u, th = zero_rest(2, n * n)
    return rho, u, th


def config_3d(n: int = 384, seed: int = 3):
    """3D: Gaussian pulse, amplitude 1e-3, width 16 cells, centre ~ U."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, n, size=3)
    rho = gaussian_pulse((n, n, n), 1e-3, 16.0, tuple(c))
    u, th = zero_rest(3, n ** 3)
    return rho, u, th


def batched_2d_specs(count: int = 96, seed: int = 4):
    """Domain list of the batched 2D workload: sizes s ~ U{128, 192, ..., 1024}, square s x s,
    pulse centre ~ U, amplitude ~ U[1e-4, 1e-3], tau ~ U[0.52, 1.2], width 16 cells."""
    rng = np.random.default_rng(seed)
    sizes = np.arange(128, 1025, 64)
    out = []
    for _ in range(count):
        s = int(rng.choice(sizes))
        out.append({"nx": s, "ny": s, "center": tuple(rng.uniform(0, s, size=2)), "amplitude": float(rng.uniform(1e-4, 1e-3)),
                    "tau": float(rng.uniform(0.52, 1.2)), "width": 16.0})
    return out


def batched_2d_fields(spec):
    rho = gaussian_pulse((spec["nx"], spec["ny"], 1), spec["amplitude"], spec["width"],
                         (spec["center"][0], spec["center"][1], 0))
    u, th = zero_rest(2, spec["nx"] * spec["ny"])
    return rho, u, th


def random_fields(shape, D: int, seed: int, scale: float = 1e-3):
    """Independent normal fields (rho', u', theta') for parity tests on arbitrary shapes."""
    rng = np.random.default_rng(seed)
    cells = int(np.prod((list(shape) + [1, 1])[:3]))
    return (scale * rng.normal(size=cells), scale * rng.normal(size=(D, cells)), scale * rng.normal(size=cells))


def random_populations(q: int, cells: int, seed: int, scale: float = 1e-3):
    rng = np.random.default_rng(seed)
    return scale * rng.normal(size=(q, cells))
