"""Two-grid convergence factor of the waveform-relaxation multigrid by mode analysis (Section 5:
semi-algebraic mode analysis -- Fourier modes in space, exact treatment in time; oracle, tests only).

The two-grid operator of one cycle with nu1 + nu2 red-black zebra-in-time sweeps, full-weighting
restriction, (bi)linear interpolation and an exact coarse solve (Algorithm 2 with two levels) acts
on the space-time error.  With homogeneous Dirichlet boundaries the sine modes of the grid are
eigenvectors of A_h, and the red-black smoother and the transfer operators couple only a mode with
its partners under n -> N+1-n in each direction: 2 modes in 1D, 4 in 2D.  On such a group every
block of the operator is a rational function of the lower-triangular time matrix R, hence lower
triangular with diagonal entries the same function of R_mm; the spectrum is therefore the union over
m of the spectra of the 2x2 (4x4) matrices obtained with R replaced by R_mm, and

    rho = max over mode groups and over m of rho(S^nu2 K S^nu1)(R_mm).

``two_grid_factor`` computes this; ``two_grid_operator`` assembles the same operator as a dense
N^dim M square matrix from the oracle's multigrid pieces (wrmg.smooth, restrict_fw, prolong, a dense
coarse solve): on small grids its mode structure and its time-diagonal blocks are the brute-force
check of the per-mode matrices (its eigenvalues themselves are ill-conditioned: the operator is far
from normal).  The mode angle is k pi / (N+1) whatever the domain length.
"""
from __future__ import annotations

import math

import numpy as np

from . import wrmg
from .direct import solve_o3


def _rho(T: np.ndarray) -> float:
    return float(np.abs(np.linalg.eigvals(T)).max())


def _group_1d(mu, c, h, nu1, nu2):
    """2x2 two-grid matrix on the amplitudes (a, b) of the modes k and N+1-k, c = cos(k pi / (N+1))."""
    s = 2.0 / h ** 2
    G = (2.0 * c / h ** 2) / (mu + s)
    # red-black smoother: odd points first; on odd points the pair reads a+b, on even ones a-b
    C = np.array([[1.0, 1.0], [1.0, -1.0]])
    S = np.linalg.solve(C, np.array([[0.0, G], [0.0, G * G]]) @ C)
    lam_k, lam_kp, lam_c = 2.0 / h ** 2 * (1 - c), 2.0 / h ** 2 * (1 + c), (1 - c * c) / h ** 2
    P = np.array([[(1 + c) / 2], [-(1 - c) / 2]])           # interpolation of the coarse mode
    Rr = P.T                                               # full weighting onto it
    A = np.diag([mu + lam_k, mu + lam_kp])
    K = np.eye(2) - P @ Rr @ A / (mu + lam_c)
    return np.linalg.matrix_power(S, nu2) @ K @ np.linalg.matrix_power(S, nu1)


def _group_2d(mu, cx, cy, h, nu1, nu2):
    """4x4 two-grid matrix on the amplitudes of the modes (k,l), (k',l'), (k',l), (k,l'),
    k' = N+1-k; cx = cos(k pi / (N+1)), cy = cos(l pi / (N+1))."""
    s = 4.0 / h ** 2
    # grid values per point class (i odd/even, j odd/even; 1-based): v = C a, C^-1 = C / 4
    C = np.array([[1, 1, 1, 1], [1, 1, -1, -1], [1, -1, 1, -1], [1, -1, -1, 1]], dtype=float)  # oo, ee, oe, eo
    g = 1.0 / (h ** 2 * (mu + s))
    # red (i + j even: oo, ee) first; x-neighbours of oo are eo, y-neighbours oe, and so on
    red = np.zeros((4, 4))
    red[0] = [0, 0, 2 * cy * g, 2 * cx * g]
    red[1] = [0, 0, 2 * cx * g, 2 * cy * g]
    red[2, 2] = red[3, 3] = 1.0
    black = np.eye(4)
    black[2] = [2 * cy * g, 2 * cx * g, 0, 0]
    black[3] = [2 * cx * g, 2 * cy * g, 0, 0]
    S = np.linalg.solve(C, black @ red @ C)
    l1 = lambda c: 2.0 / h ** 2 * (1 - c)  # noqa: E731
    lam = [l1(cx) + l1(cy), l1(-cx) + l1(-cy), l1(-cx) + l1(cy), l1(cx) + l1(-cy)]
    lam_c = (1 - cx * cx) / h ** 2 + (1 - cy * cy) / h ** 2
    Rr = np.array([[(1 + cx) * (1 + cy), (1 - cx) * (1 - cy), -(1 - cx) * (1 + cy), -(1 + cx) * (1 - cy)]]) / 4
    P = Rr.T
    K = np.eye(4) - P @ Rr @ np.diag([mu + x for x in lam]) / (mu + lam_c)
    return np.linalg.matrix_power(S, nu2) @ K @ np.linalg.matrix_power(S, nu1)


def two_grid_factor(R: np.ndarray, dim: int, N: int, h: float, nu1: int = 0, nu2: int = 1) -> float:
    """rho of the two-grid operator by mode analysis, over the paired modes k (and l) = 1..(N-1)/2."""
    mus = np.diag(R)
    ks = range(1, (N + 1) // 2)
    best = 0.0
    for k in ks:
        cx = math.cos(k * math.pi / (N + 1))
        if dim == 1:
            for mu in mus:
                best = max(best, _rho(_group_1d(mu, cx, h, nu1, nu2)))
        else:
            for l in ks:
                cy = math.cos(l * math.pi / (N + 1))
                for mu in mus:
                    best = max(best, _rho(_group_2d(mu, cx, cy, h, nu1, nu2)))
    return best


def two_grid_operator(R: np.ndarray, dim: int, N: int, h: float, nu1: int = 0, nu2: int = 1) -> np.ndarray:
    """The two-grid error propagator as a dense matrix (columns: images of unit errors), built from
    Algorithm 2's pieces with a zero right-hand side; small N^dim M only."""
    M = R.shape[0]
    shape = (M,) + (N,) * dim
    n = int(np.prod(shape))
    F = np.zeros(shape)
    T = np.empty((n, n))
    for col in range(n):
        e = np.zeros(n)
        e[col] = 1.0
        u = e.reshape(shape)
        for _ in range(nu1):
            u = wrmg.smooth(R, F, u, h)
        r = wrmg.defect(R, F, u, h)
        ec = solve_o3(R, wrmg.restrict_fw(r), 2.0 * h)
        u = u + wrmg.prolong(ec)
        for _ in range(nu2):
            u = wrmg.smooth(R, F, u, h)
        T[:, col] = u.reshape(-1)
    return T
