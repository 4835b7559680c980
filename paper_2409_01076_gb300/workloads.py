"""Seeded, synthetic input generators shared by the tests, bench.py and smoke().

This module holds problem set-up only -- initial macroscopic fields, flow
parameters, random populations and batch lists -- and none of the lattice
update's arithmetic (no equilibrium, moments, collision or streaming).  Both
the CUDA library and the CPU oracle receive what it returns as inputs.

Every generator is deterministic: random draws come from numpy's PCG64 with an
explicit seed.
"""
from __future__ import annotations

import math

import numpy as np

# bc_flags encoding of the C ABI: 2 bits per side, left, right, bottom, top.
PERIODIC, WALL, MOVING = 0, 1, 2


def bc_flags(left: int, right: int, bottom: int, top: int) -> int:
    return left | (right << 2) | (bottom << 4) | (top << 6)


CAVITY = bc_flags(WALL, WALL, WALL, MOVING)          # three resting walls, lid on top
ALL_PERIODIC = bc_flags(PERIODIC, PERIODIC, PERIODIC, PERIODIC)
COUETTE = bc_flags(PERIODIC, PERIODIC, WALL, MOVING)  # x periodic, resting floor, moving top
CHANNEL = bc_flags(PERIODIC, PERIODIC, WALL, WALL)


def cavity_tau(n: int, u_lid: float, re: float) -> float:
    """Relaxation time of a lid-driven cavity of side n at Reynolds number re.

    Re = U_lid L / nu with L = n (halfway walls lie half a link outside the
    first and last rows), and the lattice viscosity relation
    nu = (tau - 1/2) / 3 (the viscosity relation of the appendix with e = dx = 1).
    """
    nu = u_lid * n / re
    return 3.0 * nu + 0.5


def tgv_fields(n_x: int, n_y: int, u0: float, x0: int = 0, y0: int = 0,
               w: int | None = None, h: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Taylor-Green vortex on a periodic n_x x n_y lattice, node coordinate x = i.

    u = (-u0 cos(kx x) sin(ky y), u0 sin(kx x) cos(ky y)),
    rho = 1 - (3 u0^2 / 4) (cos(2 kx x) + cos(2 ky y)),  kx = 2 pi / n_x, ky = 2 pi / n_y.

    Returns (rho[h][w], u[2][h][w]) for the window of nodes i = x0 .. x0+w-1,
    j = y0 .. y0+h-1 (indices wrap periodically), FP64.
    """
    w = n_x if w is None else w
    h = n_y if h is None else h
    kx = 2.0 * math.pi / n_x
    ky = 2.0 * math.pi / n_y
    xi = np.mod(np.arange(x0, x0 + w), n_x).astype(np.float64)
    yj = np.mod(np.arange(y0, y0 + h), n_y).astype(np.float64)
    cx, sx = np.cos(kx * xi), np.sin(kx * xi)
    cy, sy = np.cos(ky * yj), np.sin(ky * yj)
    c2x, c2y = np.cos(2 * kx * xi), np.cos(2 * ky * yj)
    u = np.empty((2, h, w))
    u[0] = -u0 * np.outer(sy, cx)
    u[1] = u0 * np.outer(cy, sx)
    rho = 1.0 - 0.75 * u0 * u0 * (c2x[None, :] + c2y[:, None])
    return rho, u


def rest_fields(nx: int, ny: int) -> tuple[np.ndarray, np.ndarray]:
    """rho = 1, u = 0 everywhere (the cavity's initial state)."""
    return np.ones((ny, nx)), np.zeros((2, ny, nx))


def random_macros(nx: int, ny: int, seed: int, u_amp: float = 0.05,
                  rho_amp: float = 0.02) -> tuple[np.ndarray, np.ndarray]:
    """Smooth-free random rho in 1 +- rho_amp and u in +-u_amp (uniform), seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = 1.0 + rho_amp * rng.uniform(-1.0, 1.0, size=(ny, nx))
    u = u_amp * rng.uniform(-1.0, 1.0, size=(2, ny, nx))
    return rho, u


def random_populations(nx: int, ny: int, seed: int, lo: float = 0.02,
                       hi: float = 0.45) -> np.ndarray:
    """Positive random populations f[9][ny][nx], uniform in [lo, hi], seeded.

    Far from equilibrium on purpose: it exercises every non-equilibrium part.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(9, ny, nx))


def random_node_populations(count: int, seed: int) -> np.ndarray:
    """count x 9 positive populations near rest: w-like magnitudes times (1 + 0.1 xi).

    The magnitudes (4/9, 1/9 x4, 1/36 x4) only set a realistic scale; they are
    inputs here, not the method's weights.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return scale[None, :] * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, size=(count, 9)))


def batched_cavities(count: int = 512, seed: int = 0, sides=(64, 128, 256, 512, 1024),
                     re_lo: float = 100.0, re_hi: float = 5000.0):
    """Uneven cavity batch: sides uniform over `sides`, Re log-uniform in [re_lo, re_hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.choice(np.asarray(sides), size=count)
    re = np.exp(rng.uniform(math.log(re_lo), math.log(re_hi), size=count))
    return [(int(a), float(b)) for a, b in zip(n, re)]
