"""Pins for oracle.l1: the L1 matrix R of Eq. (elements_matrix_R), the initial-data weights,
the Mittag-Leffler series and the discretisation error of Table 1."""
import math

import mpmath
import numpy as np
import pytest

from oracle import direct, l1
from tests.conftest import load_golden


def _mp_entry(tm, tj_m1, tj, tj_p1, alpha, diag):
    """R_{m,j} from the closed-form integral of phi_j' (50-digit arithmetic, no cancellation
    issue at this precision)."""
    p = 1 - alpha
    g2 = mpmath.gamma(2 - alpha)
    rise = ((tm - tj_m1) ** p - (tm - tj) ** p) / (tj - tj_m1)
    if diag:
        return rise / g2
    fall = ((tm - tj) ** p - (tm - tj_p1) ** p) / (tj_p1 - tj)
    return (rise - fall) / g2


@pytest.mark.parametrize("alpha,gamma", [(0.3, 1.0), (0.5, 2.0), (0.8, 1.5), (0.3, 1.7 / 0.3)])
def test_R_matches_50_digit_closed_form(alpha, gamma):
    mpmath.mp.dps = 60
    M = 24
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    tm_ = [mpmath.mpf(float(v)) for v in t]       # same (double) mesh points, exact arithmetic
    a = mpmath.mpf(alpha)
    worst = 0.0
    for m in range(1, M + 1):
        for j in range(1, m + 1):
            ref = _mp_entry(tm_[m], tm_[j - 1], tm_[j], tm_[j + 1] if j < M else None, a, j == m)
            worst = max(worst, abs(float((mpmath.mpf(R[m - 1, j - 1]) - ref) / ref)))
    assert worst < 1e-12, worst


def test_uniform_mesh_is_textbook_L1():
    """On a uniform mesh R_{m,m-k} = tau^-alpha/Gamma(2-alpha) (b_k - b_{k-1}),
    b_k = (k+1)^(1-alpha) - k^(1-alpha), b_{-1} = 0 (classical L1 weights)."""
    mpmath.mp.dps = 40
    M, alpha = 40, 0.45
    t = l1.graded_mesh(2.0, M, 1.0)
    R = l1.l1_matrix(t, alpha)
    tau = mpmath.mpf(2) / M
    p = 1 - mpmath.mpf(alpha)
    b = [(k + 1) ** p - k ** p for k in range(M)]
    for m in range(1, M + 1):
        for k in range(m):
            ref = tau ** (-mpmath.mpf(alpha)) / mpmath.gamma(2 - mpmath.mpf(alpha)) * (b[k] - (b[k - 1] if k else 0))
            assert abs(R[m - 1, m - 1 - k] - float(ref)) <= 1e-13 * abs(float(ref)) + 1e-300


@pytest.mark.parametrize("alpha,gamma,M", [(0.5, 2.0, 64), (0.3, 1.7 / 0.3, 256), (0.8, 1.5, 512)])
def test_exact_on_piecewise_linear(alpha, gamma, M):
    """The L1 scheme is exact for u = 1 and u = t (both lie in the trial space):
    the discrete Caputo derivative of 1 vanishes (row sums of R equal d_{m,m}) and that of t
    equals t^(1-alpha)/Gamma(2-alpha)."""
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    dmm = l1.initial_coeff(t, alpha)
    rows = R.sum(axis=1)
    assert np.max(np.abs(rows - dmm) / dmm) < 1e-11
    lin = R @ t[1:]
    ref = t[1:] ** (1 - alpha) / math.gamma(2 - alpha)
    assert np.max(np.abs(lin - ref) / ref) < 1e-11


def test_R_sign_structure():
    """Diagonal positive, strictly lower part negative, upper part zero."""
    t = l1.graded_mesh(1.0, 128, 2.5)
    R = l1.l1_matrix(t, 0.4)
    assert np.all(np.diag(R) > 0)
    assert np.all(R[np.tril_indices(128, -1)] < 0)
    assert np.all(R[np.triu_indices(128, 1)] == 0)


def test_mittag_leffler_special_cases():
    x = np.linspace(0, 1, 11)
    assert np.allclose(l1.mittag_leffler(1.0, -x), np.exp(-x), rtol=1e-14, atol=1e-15)
    ref = np.array([float(mpmath.exp(v * v) * mpmath.erfc(v)) for v in x])
    assert np.allclose(l1.mittag_leffler(0.5, -x), ref, rtol=1e-13, atol=1e-15)
    assert np.allclose(l1.mittag_leffler(2.0, -x * x), np.cos(x), rtol=1e-14, atol=1e-15)


def test_table1_errors():
    """Table 1: max error of the L1 scheme for u = E_delta(-t^delta) sin x, N = 1024.
    The discrete solution is the mode sin(x_n) times w with (R + lam_h I) w = d_{.,m} (f = 0,
    g = sin x), lam_h = (4/h^2) sin^2(h/2), h = pi/(N+1)."""
    N = 1024
    h = math.pi / (N + 1)
    lam = 4.0 / h ** 2 * math.sin(h / 2) ** 2
    x = np.arange(1, N + 1) * h
    smax = np.sin(x).max()
    rows = load_golden("table1_errors.txt")
    got = {}
    for delta, M, E_paper in rows:
        M = int(M)
        t = l1.graded_mesh(1.0, M, (2 - delta) / delta)
        R = l1.l1_matrix(t, delta)
        w = direct.solve_o2_mode(R, lam, l1.initial_coeff(t, delta))
        exact = l1.mittag_leffler(delta, -t[1:] ** delta)
        E = np.abs(exact - w).max() * smax
        got[(delta, M)] = E
        # printed to two digits; the first column differs by up to ~6 %
        assert abs(E - E_paper) <= 0.08 * E_paper, (delta, M, E, E_paper)
    for delta in (0.4, 0.6, 0.8):
        order = math.log2(got[(delta, 256)] / got[(delta, 512)])
        assert abs(order - (2 - delta)) < 0.5 and order > 1.0


@pytest.mark.parametrize("alpha,gamma,expected", [(0.5, 2.0, 1.0), (0.3, 1.7 / 0.3, 1.7), (0.8, 1.0, 0.8)])
def test_time_convergence_rate(alpha, gamma, expected):
    """Observed order of the time error approaches min(2-alpha, gamma*alpha) for the
    typical solution t^alpha (source Gamma(1+alpha) + lam t^alpha, exact for this mode)."""
    lam = 9.0
    errs = []
    for M in (128, 256, 512, 1024):
        t = l1.graded_mesh(1.0, M, gamma)
        R = l1.l1_matrix(t, alpha)
        tt = t[1:]
        w = direct.solve_o2_mode(R, lam, math.gamma(1 + alpha) + lam * tt ** alpha)
        errs.append(np.abs(w - tt ** alpha).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert abs(rates[-1] - expected) < 0.12, rates
