"""Graded time mesh and the Petrov-Galerkin L1 matrix R (oracle; test infrastructure only).

Section 2 of Hu, Rodrigo & Gaspar defines the time discretisation of the Caputo derivative
by hat trial functions phi_j on the mesh 0 = t_0 < ... < t_M = T and Dirac test functions at
t_m.  The entries of the (lower-triangular) matrix R are the integrals of
Eq. (elements_matrix_R):

    R[m, j] = 1/Gamma(1-alpha) * int_0^{t_m} (t_m - s)^(-alpha) phi_j'(s) ds,   1 <= j <= m.

(alpha is the paper's fractional order delta.)  The mesh is t_m = T (m/M)^gamma (the paper's
grading exponent r, Section 2).

How each entry is evaluated here (no step relies on the paper's difference formulas for
d_{m,k}, which cancel catastrophically far from the diagonal):

* j >= m-2 ("near"): the integral in closed form.  phi_j' is 1/tau on the rising half of the
  hat and -1/tau on the falling half, so R[m, j] = D(m, j) - D(m, j+1) (D(m, m+1) = 0) with

      D(m, i) = [(t_m - t_{i-1})^(1-alpha) - (t_m - t_i)^(1-alpha)] / ((t_i - t_{i-1}) Gamma(2-alpha)),

  and every power difference (b + d)^p - b^p is taken as b^p * expm1(p * log1p(d / b)).
  In the paper's notation D(m, m-k+1) = d_{m,k}; R[m, m] = d_{m,1} = tau_m^(-alpha)/Gamma(2-alpha).
* j <= m-3 ("far"): integration by parts moves the derivative onto the kernel (phi_j vanishes
  at both ends of its support, which ends at t_{j+1} < t_m):

      R[m, j] = -alpha/Gamma(1-alpha) * int_{t_{j-1}}^{t_{j+1}} (t_m - s)^(-1-alpha) phi_j(s) ds,

  a positive integrand with no cancellation, evaluated by Gauss-Legendre on each half of the
  hat.  The nearest singularity is at least two mesh steps (each >= the half-interval length
  on a mesh with non-decreasing steps) away, so 24 nodes reach full double precision.

Initial data (paper: u(x, 0) = g, Eq. discrete_model_IVP_3): the coefficient of u_0 in the
discrete Caputo derivative at t_m is -D(m, 1) = -d_{m,m}; moved to the right-hand side it adds
d_{m,m} * g.
"""
from __future__ import annotations

import math

import numpy as np

NQ_DEFAULT = 24


def graded_mesh(T: float, M: int, gamma: float) -> np.ndarray:
    """t_m = T (m/M)^gamma, m = 0..M (Section 2; gamma is the paper's r)."""
    m = np.arange(M + 1, dtype=np.float64)
    return T * (m / M) ** gamma


def _pow_step(b: np.ndarray, d: np.ndarray, p: float) -> np.ndarray:
    """(b + d)^p - b^p for b >= 0, d > 0, without cancellation."""
    b = np.asarray(b, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    out = np.empty(np.broadcast(b, d).shape)
    bb, dd = np.broadcast_arrays(b, d)
    pos = bb > 0
    out[pos] = bb[pos] ** p * np.expm1(p * np.log1p(dd[pos] / bb[pos]))
    out[~pos] = dd[~pos] ** p
    return out


def _D(t: np.ndarray, alpha: float, m: int, i: np.ndarray) -> np.ndarray:
    """D(m, i) for 1 <= i <= m (see module docstring); equals the paper's d_{m, m-i+1}."""
    p = 1.0 - alpha
    b = t[m] - t[i]
    tau = t[i] - t[i - 1]
    return _pow_step(b, tau, p) / (tau * math.gamma(2.0 - alpha))


def l1_matrix(t: np.ndarray, alpha: float, nq: int = NQ_DEFAULT) -> np.ndarray:
    """Dense M x M lower-triangular R with R[m-1, j-1] = R_{m,j} (Eq. elements_matrix_R)."""
    M = len(t) - 1
    R = np.zeros((M, M))
    xg, wg = np.polynomial.legendre.leggauss(nq)
    left_shape = 0.5 * (1.0 + xg)       # phi_j on the rising half, at the nodes
    right_shape = 0.5 * (1.0 - xg)      # phi_j on the falling half, at the nodes
    far_scale = -alpha / math.gamma(1.0 - alpha)
    for m in range(1, M + 1):
        # near entries, closed form
        R[m - 1, m - 1] = (t[m] - t[m - 1]) ** (-alpha) / math.gamma(2.0 - alpha)
        for j in range(max(1, m - 2), m):
            Dj = _D(t, alpha, m, np.array([j]))[0]
            Dj1 = _D(t, alpha, m, np.array([j + 1]))[0]
            R[m - 1, j - 1] = Dj - Dj1
        if m <= 3:
            continue
        # far entries j = 1..m-3, integration by parts + Gauss-Legendre
        j = np.arange(1, m - 2)
        tau_l = t[j] - t[j - 1]
        tau_r = t[j + 1] - t[j]
        # distance from t_m to the nodes of each half: t_m - s
        dl = (t[m] - t[j - 1])[:, None] - tau_l[:, None] * left_shape[None, :]
        dr = (t[m] - t[j])[:, None] - tau_r[:, None] * left_shape[None, :]
        il = 0.5 * tau_l * ((dl ** (-1.0 - alpha)) * left_shape[None, :] * wg[None, :]).sum(axis=1)
        ir = 0.5 * tau_r * ((dr ** (-1.0 - alpha)) * right_shape[None, :] * wg[None, :]).sum(axis=1)
        R[m - 1, j - 1] = far_scale * (il + ir)
    return R


def initial_coeff(t: np.ndarray, alpha: float) -> np.ndarray:
    """d_{m,m} = D(m, 1) for m = 1..M: the weight of g = u(., 0) on the right-hand side."""
    M = len(t) - 1
    return np.array([_D(t, alpha, m, np.array([1]))[0] for m in range(1, M + 1)])


def mittag_leffler(alpha: float, z: np.ndarray, terms: int = 400) -> np.ndarray:
    """E_alpha(z) = sum_k z^k / Gamma(alpha k + 1) (Section 5.1), for |z| <= 1."""
    z = np.asarray(z, dtype=np.float64)
    out = np.zeros_like(z)
    for k in range(terms):
        out += z ** k * math.exp(-math.lgamma(alpha * k + 1.0))
    return out
