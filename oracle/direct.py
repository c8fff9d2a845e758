"""Direct solvers for the fully discrete problem (oracle; test infrastructure only).

The discrete problem of Section 2, Eqs. (discrete_model_IVP_1-3), written with a dense
lower-triangular time matrix R (R[m-1, j-1] = R_{m,j}) and the initial-data weights
dmm[m-1] = d_{m,m}:

    sum_{j<=m} R_{m,j} u_{n,j} + (A_h u_{., m})_n = f(x_n, t_m) + d_{m,m} g(x_n),

for every interior point n and every time level m = 1..M, with homogeneous Dirichlet
boundaries.  A_h is the 3-point (1D) or 5-point (2D) negative Laplacian with grid size
h = L/(N+1) per dimension (Eq. discrete_model_IVP_1 and Section 5.2).

Arrays are time-major, space contiguous: u[m-1, n-1] (1D) or u[m-1, iy, ix] (2D).

* ``solve_o1`` -- implicit time stepping: at each m, move the known history sum
  sum_{j<m} R_{m,j} u_j to the right-hand side and solve (R_{m,m} I + A_h) u_m = rhs; the
  spatial solve is a tridiagonal banded solve (1D) or the DST-I diagonalisation of the
  5-point Laplacian (2D).
* ``solve_o2_mode`` -- when the data are one sine mode sin(k pi x)[sin(l pi y)], which is an
  exact eigenvector of A_h with eigenvalue lam, the solution is that mode times w with
  (R + lam I) w = F (one M x M lower-triangular solve).
* ``solve_o3`` -- assembles the whole N^dim M x N^dim M matrix kron(R, I) + kron(I, A_h) and
  solves it densely (tiny sizes only).
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.linalg


def laplacian_eigs_1d(N: int, h: float) -> np.ndarray:
    """Eigenvalues (4/h^2) sin^2(p pi h' / 2), p = 1..N, of the 3-point -d^2/dx^2 with
    N interior points (eigenvector sin(p pi n / (N+1)))."""
    p = np.arange(1, N + 1)
    return 4.0 / h ** 2 * np.sin(p * np.pi / (2.0 * (N + 1))) ** 2


def apply_ah(u: np.ndarray, h: float) -> np.ndarray:
    """A_h u for a batch of grid functions u[..., n] (1D) or u[..., iy, ix] (2D is chosen by
    calling apply_ah_2d); zero Dirichlet boundaries."""
    up = np.zeros(u.shape[:-1] + (u.shape[-1] + 2,))
    up[..., 1:-1] = u
    return (2.0 * u - up[..., :-2] - up[..., 2:]) / h ** 2


def apply_ah_2d(u: np.ndarray, h: float) -> np.ndarray:
    """5-point negative Laplacian on u[..., iy, ix] with zero Dirichlet boundaries."""
    up = np.zeros(u.shape[:-2] + (u.shape[-2] + 2, u.shape[-1] + 2))
    up[..., 1:-1, 1:-1] = u
    return (4.0 * u - up[..., :-2, 1:-1] - up[..., 2:, 1:-1] - up[..., 1:-1, :-2] - up[..., 1:-1, 2:]) / h ** 2


def rhs_with_initial(f: np.ndarray, dmm: np.ndarray, g: np.ndarray | None) -> np.ndarray:
    """F = f + d_{m,m} g (the initial value u_0 = g moved to the right-hand side)."""
    if g is None:
        return np.array(f, dtype=np.float64, copy=True)
    return f + dmm.reshape((-1,) + (1,) * (f.ndim - 1)) * g[None, ...]


def residual(R: np.ndarray, F: np.ndarray, u: np.ndarray, h: float) -> np.ndarray:
    """r = F - (R (x) I) u - (I (x) A_h) u  (the defect of Algorithm 2)."""
    M = R.shape[0]
    Ru = (R @ u.reshape(M, -1)).reshape(u.shape)
    Au = apply_ah(u, h) if u.ndim == 2 else apply_ah_2d(u, h)
    return F - Ru - Au


def solve_o1(R: np.ndarray, F: np.ndarray, h: float, m_stop: int | None = None) -> np.ndarray:
    """Implicit time stepping with the dense history sum (the direct oracle).

    F is the full right-hand side (f + d_{m,m} g), shape (M, N) or (M, N, N).  If m_stop is
    given only the first m_stop time levels are computed (a bounded sample for timing)."""
    M = R.shape[0]
    steps = M if m_stop is None else min(M, m_stop)
    u = np.zeros_like(F, dtype=np.float64)
    flat_u = u.reshape(M, -1)
    flat_F = F.reshape(M, -1)
    dim = F.ndim - 1
    N = F.shape[-1]
    if dim == 1:
        ab = np.zeros((3, N))
        ab[0, 1:] = -1.0 / h ** 2
        ab[2, :-1] = -1.0 / h ** 2
    else:
        lam = laplacian_eigs_1d(N, h)
        lam2 = lam[:, None] + lam[None, :]
    for m in range(steps):
        rhs = flat_F[m] - R[m, :m] @ flat_u[:m] if m else flat_F[m].copy()
        if dim == 1:
            ab[1, :] = R[m, m] + 2.0 / h ** 2
            flat_u[m] = scipy.linalg.solve_banded((1, 1), ab, rhs)
        else:
            rh = scipy.fft.dstn(rhs.reshape(N, N), type=1)
            flat_u[m] = scipy.fft.idstn(rh / (R[m, m] + lam2), type=1).reshape(-1)
    return u


def solve_o2_mode(R: np.ndarray, lam: float, Ft: np.ndarray) -> np.ndarray:
    """(R + lam I) w = Ft for one spatial eigenmode with eigenvalue lam."""
    return scipy.linalg.solve_triangular(R + lam * np.eye(R.shape[0]), Ft, lower=True)


def solve_o3(R: np.ndarray, F: np.ndarray, h: float) -> np.ndarray:
    """Dense solve of kron(R, I) + kron(I, A_h) (brute force; N^dim * M <= a few thousand)."""
    M = R.shape[0]
    shape = F.shape[1:]
    n = int(np.prod(shape))
    if len(shape) == 1:
        A = (np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)) / h ** 2
    else:
        N = shape[0]
        T1 = np.diag(np.full(N, 2.0)) - np.diag(np.ones(N - 1), 1) - np.diag(np.ones(N - 1), -1)
        A = (np.kron(np.eye(N), T1) + np.kron(T1, np.eye(N))) / h ** 2
    big = np.kron(R, np.eye(n)) + np.kron(np.eye(M), A)
    return np.linalg.solve(big, F.reshape(-1)).reshape(F.shape)
