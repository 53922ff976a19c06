"""Seeded synthetic inputs for the 7-point smoothers.

This module only draws numbers; it holds none of the smoothers' arithmetic,
so the CUDA path, the tests and the CPU oracle can all take their inputs from
it.  Arrays are numpy, shape ``(nz+2, ny+2, nx+2)`` (C order, ``u[k][j][i]``,
``i`` fastest) including the one-cell Dirichlet halo.

Recipes (the paper's own workloads are FP64 boxes of 100x50x50, 400x200x200
and 200^3, Sec. 3 and Sec. 4; these are synthetic stand-ins of the same kind,
scaled so one array is far larger than the GPU's last-level cache):

* ``laplace_64``: 64^3 interior, halo U[0,1) from seed 0, interior 0, f = 0.
* ``laplace_cube(n, seed_halo=1, seed_interior=2)``: n^3, halo U[0,1),
  interior U[0,1) (400^3 is the main benchmark grid).
* ``batched_poisson``: 256 grids, each extent a multiple of 16 in [32, 192]
  drawn uniformly (seed 3), f ~ N(0,1), zero Dirichlet, u = 0,
  h = 1/(max(nx,ny,nz)+1).
* ``sine_modes_problem``: f = sum of 8 discrete sine modes with N(0,1)
  amplitudes plus N(0, 1e-3) noise (seed 4), zero Dirichlet, u = 0.
* ``served_stream``: Poisson arrivals, cube sides log-uniform in [32, 384],
  10-200 sweeps or a solve request, FP64/FP32 mix (seed 5).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def padded_shape(nx: int, ny: int, nz: int) -> tuple[int, int, int]:
    return (nz + 2, ny + 2, nx + 2)


def grid_h(nx: int, ny: int, nz: int) -> float:
    """Mesh width for a grid: h = 1/(max extent + 1) (isotropic)."""
    return 1.0 / (max(nx, ny, nz) + 1)


def halo_and_interior(nx: int, ny: int, nz: int, seed_halo: int, seed_interior: int | None,
                      dtype=np.float64) -> np.ndarray:
    """Whole padded array U[0,1) from ``seed_halo``; interior then overwritten by
    U[0,1) from ``seed_interior`` (or zeros if None).  Drawn in FP64, then cast."""
    shape = padded_shape(nx, ny, nz)
    u = np.random.default_rng(seed_halo).random(shape)
    if seed_interior is None:
        u[1:-1, 1:-1, 1:-1] = 0.0
    else:
        u[1:-1, 1:-1, 1:-1] = np.random.default_rng(seed_interior).random((nz, ny, nx))
    return np.ascontiguousarray(u.astype(dtype))


def laplace_64(dtype=np.float64) -> np.ndarray:
    return halo_and_interior(64, 64, 64, 0, None, dtype)


def laplace_cube(n: int, seed_halo: int = 1, seed_interior: int = 2, dtype=np.float64) -> np.ndarray:
    return halo_and_interior(n, n, n, seed_halo, seed_interior, dtype)


def random_grid(nx: int, ny: int, nz: int, seed: int, dtype=np.float64, with_f: bool = False):
    """Halo and interior U[0,1) from one seed; optional f ~ N(0,1) (halo of f zero)."""
    rng = np.random.default_rng(seed)
    u = rng.random(padded_shape(nx, ny, nz))
    f = None
    if with_f:
        f = np.zeros(padded_shape(nx, ny, nz))
        f[1:-1, 1:-1, 1:-1] = rng.standard_normal((nz, ny, nx))
        f = np.ascontiguousarray(f.astype(dtype))
    return np.ascontiguousarray(u.astype(dtype)), f


@dataclass
class GridCase:
    nx: int
    ny: int
    nz: int
    h: float
    u: np.ndarray
    f: np.ndarray


def batched_dims(count: int = 256, seed: int = 3, lo: int = 32, hi: int = 192, step: int = 16):
    rng = np.random.default_rng(seed)
    choices = np.arange(lo, hi + 1, step)
    return [tuple(int(x) for x in rng.choice(choices, size=3)) for _ in range(count)]


def batched_poisson(count: int = 256, seed: int = 3, lo: int = 32, hi: int = 192, step: int = 16,
                    dtype=np.float64, dims=None) -> list[GridCase]:
    """Independent Poisson grids: f ~ N(0,1) on the interior, zero Dirichlet, u = 0."""
    dims = dims if dims is not None else batched_dims(count, seed, lo, hi, step)
    rng = np.random.default_rng(seed + 1000)
    out = []
    for (nx, ny, nz) in dims:
        u = np.zeros(padded_shape(nx, ny, nz), dtype=dtype)
        f = np.zeros(padded_shape(nx, ny, nz), dtype=dtype)
        f[1:-1, 1:-1, 1:-1] = rng.standard_normal((nz, ny, nx)).astype(dtype)
        out.append(GridCase(nx, ny, nz, grid_h(nx, ny, nz), u, f))
    return out


@dataclass
class SineProblem:
    n: int
    h: float
    modes: np.ndarray       # (8, 3) integer (p, q, r)
    amplitudes: np.ndarray  # (8,)
    noise_sigma: float
    f: np.ndarray


def sine_modes_problem(n: int, seed: int = 4, nmodes: int = 8, max_mode: int = 16,
                       noise_sigma: float = 1e-3) -> SineProblem:
    """f = sum_m a_m sin(p pi i h) sin(q pi j h) sin(r pi k h) + N(0, noise^2),
    i, j, k = 1..n the interior's 1-based indices, h = 1/(n+1); modes drawn
    uniformly from [1, max_mode]^3, a_m ~ N(0,1).  Zero Dirichlet."""
    rng = np.random.default_rng(seed)
    modes = rng.integers(1, max_mode + 1, size=(nmodes, 3))
    amps = rng.standard_normal(nmodes)
    h = 1.0 / (n + 1)
    idx = np.arange(1, n + 1, dtype=np.float64)
    f = np.zeros((n + 2, n + 2, n + 2))
    inner = np.zeros((n, n, n))
    for (p, q, r), a in zip(modes, amps):
        sx = np.sin(p * np.pi * idx * h)
        sy = np.sin(q * np.pi * idx * h)
        sz = np.sin(r * np.pi * idx * h)
        inner += a * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    if noise_sigma > 0:
        inner += noise_sigma * rng.standard_normal((n, n, n))
    f[1:-1, 1:-1, 1:-1] = inner
    return SineProblem(n, h, modes, amps, noise_sigma, np.ascontiguousarray(f))


@dataclass
class Request:
    arrival_s: float
    n: int              # cube side
    kind: str           # "jacobi" | "gs" | "solve"
    sweeps: int         # sweeps for jacobi/gs; sweep cap for solve
    dtype: str          # "f64" | "f32"
    rtol: float
    seed: int


def served_stream(rate_hz: float, count: int, seed: int = 5, lo: int = 32, hi: int = 384,
                  solve_fraction: float = 0.2, f32_fraction: float = 0.5,
                  solve_cap: int = 2000) -> list[Request]:
    """Poisson arrivals at ``rate_hz``; cube side log-uniform in [lo, hi];
    10-200 sweeps of Jacobi or GS, or a solve to 1e-8 capped at ``solve_cap`` sweeps."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
    out = []
    for m in range(count):
        n = int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))
        u = rng.random()
        if u < solve_fraction:
            kind, sweeps = "solve", solve_cap
        else:
            kind = "jacobi" if rng.random() < 0.5 else "gs"
            sweeps = int(rng.integers(10, 201))
        dt = "f32" if rng.random() < f32_fraction else "f64"
        out.append(Request(float(t[m]), n, kind, sweeps, dt, 1e-8, int(rng.integers(0, 2**31 - 1))))
    return out
