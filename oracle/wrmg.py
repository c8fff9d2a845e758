"""Algorithm 2 -- multigrid waveform relaxation, plain recursive form (oracle; tests only).

The space-time operator on a level with N interior points per dimension and grid size h is
A_{h,tau} = Rt (x) I + I (x) A_h, where Rt is the time matrix (the dense L1 matrix R, or its
H-approximation R~ returned densely by ``oracle.hmatrix``); the same Rt is used on every
level because the coarsening is in space only (Algorithm 2).  Steps of one cycle, in the
paper's order:

1. nu1 pre-smoothing steps of zebra-in-time line relaxation: red-black Gauss-Seidel in space
   where each update solves a whole time line, (Rt + s I) u_n = F_n + (sum of the
   neighbours' time lines)/h^2, s = 2/h^2 (1D) or 4/h^2 (2D) (Section 4, relaxation step).
   Colour order (Section 4 updates "the even points" first): the paper's numbering is read
   as the one that gives the boundary point x_0 the number 1, so in 1D the first colour is
   the odd interior points n = 1, 3, ... (the points that are not on the coarse grid) and
   then the even n; in 2D the first colour is the points with i + j even.  This reading
   reproduces the measured W-cycle factors of Table 2 and the V(0,1) ~ W behaviour the
   paper reports; the other order gives V(0,1) factors near 0.2.
2. defect r = F - A_{h,tau} u.
3. full-weighting restriction in space only: [1 2 1]/4 (1D), [1 2 1; 2 4 2; 1 2 1]/16 (2D);
   coarse point i sits on fine point 2i.
4. coarse-grid correction started from the zero grid function, gamma_c cycles (1 = V).
5. linear (1D) / bilinear (2D) interpolation in space only, added to u.
6. nu2 post-smoothing steps.
On the coarsest level (one interior point per dimension) the system is solved directly.
Optionally (n_direct > 1, a choice the paper leaves open: it recurses to one point) the
coarse-grid correction is solved exactly as soon as the coarse grid has at most n_direct
interior points per dimension (``direct_level_solve``); n_direct = 1 is the paper's cycle.
Line solves and products use the dense Rt (library triangular solve / matmul), which is what
Algorithms 3 and 4 compute.
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.linalg

from .direct import apply_ah, apply_ah_2d, laplacian_eigs_1d, solve_o2_mode


def _colour_masks_1d(N):
    n = np.arange(1, N + 1)
    return [n % 2 == 1, n % 2 == 0]


def _colour_masks_2d(N):
    i = np.arange(1, N + 1)
    s = i[:, None] + i[None, :]
    return [(s % 2 == 0), (s % 2 == 1)]


def _neighbour_sum(u: np.ndarray) -> np.ndarray:
    if u.ndim == 2:
        up = np.zeros((u.shape[0], u.shape[1] + 2))
        up[:, 1:-1] = u
        return up[:, :-2] + up[:, 2:]
    up = np.zeros((u.shape[0], u.shape[1] + 2, u.shape[2] + 2))
    up[:, 1:-1, 1:-1] = u
    return up[:, :-2, 1:-1] + up[:, 2:, 1:-1] + up[:, 1:-1, :-2] + up[:, 1:-1, 2:]


def diag_shift(dim: int, h: float) -> float:
    return (2.0 if dim == 1 else 4.0) / h ** 2


def smooth(Rt: np.ndarray, F: np.ndarray, u: np.ndarray, h: float) -> np.ndarray:
    """One red-black zebra-in-time sweep; returns the updated u (a new array)."""
    u = u.copy()
    dim = u.ndim - 1
    N = u.shape[1]
    masks = _colour_masks_1d(N) if dim == 1 else _colour_masks_2d(N)
    Ls = Rt + diag_shift(dim, h) * np.eye(Rt.shape[0])
    for mask in masks:
        nb = _neighbour_sum(u)
        B = F[:, mask] + nb[:, mask] / h ** 2
        u[:, mask] = scipy.linalg.solve_triangular(Ls, B, lower=True)
    return u


def defect(Rt: np.ndarray, F: np.ndarray, u: np.ndarray, h: float) -> np.ndarray:
    M = Rt.shape[0]
    Au = apply_ah(u, h) if u.ndim == 2 else apply_ah_2d(u, h)
    return F - (Rt @ u.reshape(M, -1)).reshape(u.shape) - Au


def restrict_fw(r: np.ndarray) -> np.ndarray:
    if r.ndim == 2:
        return 0.25 * (r[:, 0:-2:2] + 2.0 * r[:, 1:-1:2] + r[:, 2::2])
    rx = 0.25 * (r[:, :, 0:-2:2] + 2.0 * r[:, :, 1:-1:2] + r[:, :, 2::2])
    return 0.25 * (rx[:, 0:-2:2, :] + 2.0 * rx[:, 1:-1:2, :] + rx[:, 2::2, :])


def prolong(ec: np.ndarray) -> np.ndarray:
    if ec.ndim == 2:
        M, Nc = ec.shape
        ef = np.zeros((M, 2 * Nc + 1))
        ep = np.zeros((M, Nc + 2))
        ep[:, 1:-1] = ec
        ef[:, 1::2] = ec
        ef[:, 0::2] = 0.5 * (ep[:, :-1] + ep[:, 1:])
        return ef
    M, Nc, _ = ec.shape
    # interpolate along x, then along y (bilinear = tensor product of linear)
    tmp = np.zeros((M, Nc, 2 * Nc + 1))
    ep = np.zeros((M, Nc, Nc + 2))
    ep[:, :, 1:-1] = ec
    tmp[:, :, 1::2] = ec
    tmp[:, :, 0::2] = 0.5 * (ep[:, :, :-1] + ep[:, :, 1:])
    ef = np.zeros((M, 2 * Nc + 1, 2 * Nc + 1))
    tp = np.zeros((M, Nc + 2, 2 * Nc + 1))
    tp[:, 1:-1, :] = tmp
    ef[:, 1::2, :] = tmp
    ef[:, 0::2, :] = 0.5 * (tp[:, :-1, :] + tp[:, 1:, :])
    return ef


def coarsest_solve(Rt: np.ndarray, F: np.ndarray, h: float) -> np.ndarray:
    """Direct solve on one interior point: (Rt + s I) u = F."""
    dim = F.ndim - 1
    Ls = Rt + diag_shift(dim, h) * np.eye(Rt.shape[0])
    M = Rt.shape[0]
    return scipy.linalg.solve_triangular(Ls, F.reshape(M, -1), lower=True).reshape(F.shape)


def direct_level_solve(Rt: np.ndarray, F: np.ndarray, h: float) -> np.ndarray:
    """Exact solve of (Rt (x) I + I (x) A_h) u = F on one level.  The sine functions
    sin(p pi n / (N+1)) are the eigenvectors of A_h (eigenvalues ``laplacian_eigs_1d``; in 2D
    products of them, eigenvalue lam_p + lam_q), so the orthonormal DST-I in space decouples the
    system into one lower-triangular time system (Rt + lam I) w = F^ per spatial mode."""
    M = Rt.shape[0]
    dim = F.ndim - 1
    N = F.shape[1]
    lam = laplacian_eigs_1d(N, h)
    axes = tuple(range(1, dim + 1))
    Fh = scipy.fft.dstn(F, type=1, axes=axes, norm="ortho").reshape(M, -1)
    lam_modes = lam if dim == 1 else (lam[:, None] + lam[None, :]).reshape(-1)
    W = np.empty_like(Fh)
    for k, lk in enumerate(lam_modes):
        W[:, k] = solve_o2_mode(Rt, lk, Fh[:, k])
    return scipy.fft.idstn(W.reshape(F.shape), type=1, axes=axes, norm="ortho")


def cycle(Rt, F, u, h, nu1=1, nu2=1, gamma_c=1, n_direct=1):
    """One WRMG cycle of Algorithm 2 on the level of F (V-cycle for gamma_c = 1).  The
    coarse-grid correction is solved exactly once the coarse grid has <= n_direct points per
    dimension (n_direct = 1: the paper's recursion to one point)."""
    N = F.shape[1]
    if N == 1:
        return coarsest_solve(Rt, F, h)
    for _ in range(nu1):
        u = smooth(Rt, F, u, h)
    r = defect(Rt, F, u, h)
    rc = restrict_fw(r)
    if n_direct > 1 and rc.shape[1] <= n_direct:
        ec = direct_level_solve(Rt, rc, 2.0 * h)
    else:
        ec = np.zeros_like(rc)
        for _ in range(gamma_c):
            ec = cycle(Rt, rc, ec, 2.0 * h, nu1, nu2, gamma_c, n_direct)
    u = u + prolong(ec)
    for _ in range(nu2):
        u = smooth(Rt, F, u, h)
    return u


def solve(Rt, F, h, nu1=1, nu2=1, rtol=1e-10, max_cycles=50, gamma_c=1, u0=None, n_direct=1):
    """Cycles from u0 (default zero) until ||r_k||_inf <= rtol ||r_0||_inf.
    Returns (u, cycles, residual-norm history)."""
    u = np.zeros_like(F) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
    hist = [np.abs(defect(Rt, F, u, h)).max()]
    k = 0
    while hist[-1] > rtol * hist[0] and k < max_cycles:
        u = cycle(Rt, F, u, h, nu1, nu2, gamma_c, n_direct)
        hist.append(np.abs(defect(Rt, F, u, h)).max())
        k += 1
    return u, k, hist
