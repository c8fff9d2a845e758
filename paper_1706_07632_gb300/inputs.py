"""Seeded synthetic inputs (sources, initial data) shared by the tests and the benchmark.

This module holds none of the solver's arithmetic: it only evaluates given source terms at
given points.  The time levels t_1..t_M are passed in by the caller (from the library's mesh or
the oracle's), and every random draw comes from numpy.random.default_rng(seed).

Workloads (sizes and distributions follow the configurations the benchmark runs):
* manufactured:  u = t^alpha sin(pi x) [sin(pi y)] on (0,1)^dim, whose Caputo derivative is
  Gamma(1+alpha), so f = (Gamma(1+alpha) + dim pi^2 t^alpha) prod sin(pi x_i), g = 0.
* sine_series_1d: f(x, t) = sum_{k=1..8} c_k / k^2 sin(k pi x), c_k ~ N(0, 1), constant in t.
* grf_2d:        f(x, y, t) = sum_{p,q} c_pq sin(p pi x) sin(q pi y), constant in t, with
  c_pq ~ N(0, exp(-(pi ell)^2 (p^2 + q^2) / 2)) (squared-exponential spectrum, length scale
  ell), truncated where the variance drops below 1e-12 of its maximum.
* mittag_leffler_1d: f = 0, g = sin(x) on (0, pi) (the 1D experiment of Section 5.1).
Each returns separable factors (time profile, spatial profile) so that large fields can be
formed on the device as an outer product.
"""
from __future__ import annotations

import math

import numpy as np


def grid(N: int, Lx: float = 1.0) -> np.ndarray:
    """Interior points x_n = n h, h = Lx/(N+1), n = 1..N."""
    return np.arange(1, N + 1) * (Lx / (N + 1))


def manufactured(t: np.ndarray, N: int, dim: int, alpha: float):
    """(a(t), s(x)) with f = a(t) s(x): a = Gamma(1+alpha) + dim pi^2 t^alpha, s = prod sin(pi x)."""
    x = grid(N)
    s = np.sin(math.pi * x)
    if dim == 2:
        s = np.outer(s, s)
    a = math.gamma(1 + alpha) + dim * math.pi ** 2 * np.asarray(t) ** alpha
    return a, s


def manufactured_exact(t: np.ndarray, N: int, dim: int, alpha: float) -> np.ndarray:
    """u(x, t) = t^alpha prod sin(pi x) at the grid points, shape (M, N[, N])."""
    a = np.asarray(t) ** alpha
    x = grid(N)
    s = np.sin(math.pi * x)
    if dim == 2:
        s = np.outer(s, s)
    return a.reshape((-1,) + (1,) * dim) * s[None]


def sine_series_1d(seed: int, t: np.ndarray, N: int, modes: int = 8):
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(modes)
    x = grid(N)
    k = np.arange(1, modes + 1)
    s = (c[:, None] / k[:, None] ** 2 * np.sin(math.pi * k[:, None] * x[None, :])).sum(axis=0)
    return np.ones(len(t)), s, c


def grf_2d(seed: int, t: np.ndarray, N: int, ell: float = 0.1):
    rng = np.random.default_rng(seed)
    kmax = 1
    while math.exp(-(math.pi * ell) ** 2 * (kmax + 1) ** 2 / 2) > 1e-12 and kmax < N:
        kmax += 1
    p = np.arange(1, kmax + 1)
    var = np.exp(-(math.pi * ell) ** 2 * (p[:, None] ** 2 + p[None, :] ** 2) / 2)
    var = var / var.max()
    c = rng.standard_normal((kmax, kmax)) * np.sqrt(var) * (var >= 1e-12)
    x = grid(N)
    S = np.sin(math.pi * np.outer(p, x))       # (kmax, N)
    s = S.T @ c @ S                              # s[iy, ix] = sum c_pq sin(p pi y) sin(q pi x)
    return np.ones(len(t)), s, c


def mittag_leffler_1d(N: int):
    """f = 0, g = sin(x) on (0, pi): returns (g, Lx)."""
    x = grid(N, math.pi)
    return np.sin(x), math.pi


def random_field(seed: int, shape) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)
