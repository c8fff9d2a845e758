"""Pins for oracle.direct, oracle.hmatrix and oracle.wrmg: brute force on tiny inputs,
eigenmode solutions, spatial order, the Theorem 3.1 bound, the printed B closed form, and the
multigrid factors / cycle counts of Tables 2, 3 and 5."""
import math

import mpmath
import numpy as np
import pytest

from oracle import direct, hmatrix, l1, wrmg
from tests.conftest import load_golden


def _manufactured(dim, N, M, alpha, gamma):
    t = l1.graded_mesh(1.0, M, gamma)
    h = 1.0 / (N + 1)
    x = np.arange(1, N + 1) * h
    amp = math.gamma(1 + alpha) + dim * math.pi ** 2 * t[1:] ** alpha
    S = np.sin(math.pi * x)
    if dim == 2:
        S = S[:, None] * S[None, :]
    F = amp.reshape((-1,) + (1,) * dim) * S[None]
    return t, h, F


@pytest.mark.parametrize("dim,N,M", [(1, 7, 12), (1, 15, 8), (2, 3, 10), (2, 7, 4)])
def test_o1_matches_brute_force(dim, N, M):
    alpha, gamma = 0.6, 1.8
    t, h, F = _manufactured(dim, N, M, alpha, gamma)
    rng = np.random.default_rng(3)
    F = F + rng.standard_normal(F.shape)          # break the single-mode structure
    g = rng.standard_normal(F.shape[1:])
    R = l1.l1_matrix(t, alpha)
    Fg = direct.rhs_with_initial(F, l1.initial_coeff(t, alpha), g)
    u1 = direct.solve_o1(R, Fg, h)
    u3 = direct.solve_o3(R, Fg, h)
    assert np.abs(u1 - u3).max() <= 1e-12 * np.abs(u3).max()
    assert np.abs(direct.residual(R, Fg, u1, h)).max() <= 1e-10 * np.abs(Fg).max()


@pytest.mark.parametrize("dim,N,M", [(1, 63, 64), (2, 15, 32)])
def test_o1_matches_o2_single_mode(dim, N, M):
    alpha, gamma = 0.5, 2.0
    t, h, F = _manufactured(dim, N, M, alpha, gamma)
    R = l1.l1_matrix(t, alpha)
    u1 = direct.solve_o1(R, F, h)
    lam = dim * 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    amp = math.gamma(1 + alpha) + dim * math.pi ** 2 * t[1:] ** alpha
    w = direct.solve_o2_mode(R, lam, amp)
    x = np.arange(1, N + 1) * h
    S = np.sin(math.pi * x)
    if dim == 2:
        S = S[:, None] * S[None, :]
    u2 = w.reshape((-1,) + (1,) * dim) * S[None]
    assert np.abs(u1 - u2).max() <= 1e-12 * np.abs(u2).max()


def test_laplacian_eigs_are_eigenvalues():
    N, h = 9, 0.1
    lam = direct.laplacian_eigs_1d(N, h)
    x = np.arange(1, N + 1)
    for p in (1, 4, 9):
        v = np.sin(p * math.pi * x / (N + 1))
        assert np.allclose(direct.apply_ah(v[None], h)[0], lam[p - 1] * v, rtol=1e-13, atol=1e-10)


def test_spatial_order_two():
    """Error against u = t^alpha sin(pi x) at fixed fine M: the spatial part is O(h^2)."""
    alpha, gamma, M = 0.5, 2.0, 64
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    amp_src = math.gamma(1 + alpha) + math.pi ** 2 * t[1:] ** alpha
    errs = []
    for N in (7, 15, 31):
        h = 1.0 / (N + 1)
        lam = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
        w_h = direct.solve_o2_mode(R, lam, amp_src)
        w_0 = direct.solve_o2_mode(R, math.pi ** 2, amp_src)   # same time scheme, exact in space
        errs.append(np.abs(w_h - w_0).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - 2.0) < 0.05 for r in rates), rates


# ---------------------------------------------------------------- H-matrix (Section 3)

def test_block_tree_partitions_matrix():
    M, leaf = 256, 16
    t = l1.graded_mesh(1.0, M, 2.5)
    cover = np.zeros((M, M), dtype=int)
    for b in hmatrix.block_tree(t, leaf):
        cover[b.r0:b.r1, b.c0:b.c1] += 1
        if b.kind == "zero":
            assert b.c0 >= b.r1
        if b.r0 == b.c0:
            assert b.kind == "dense"                 # diagonal blocks are never admissible
        if b.kind == "rk":
            assert b.c1 <= b.r0                      # strictly below the diagonal
    assert np.all(cover == 1)


def test_B_matches_printed_closed_form_50_digits():
    """Eq. (B_elements): B_{j,nu} = c_nu/(1-delta-nu) [(m_{j-1}-m_j)/tau_{j-1} - (m_j-m_{j+1})/tau_j],
    m_i = (t_0 - t_i)^(1-delta-nu), evaluated with 60 digits, against the oracle's
    integrated-by-parts quadrature (scaled by rho^nu)."""
    mpmath.mp.dps = 60
    M, leaf, alpha, k = 128, 8, 0.35, 10
    t = l1.graded_mesh(1.0, M, 1.65 / 0.35)
    rk = [b for b in hmatrix.block_tree(t, leaf) if b.kind == "rk"]
    assert rk
    for blk in rk[:: max(1, len(rk) // 8)]:
        A, B = hmatrix.rk_factors(t, alpha, blk, k)
        a, b = mpmath.mpf(float(t[blk.r0 + 1])), mpmath.mpf(float(t[blk.r1]))
        tc = (a + b) / 2
        rho = (b - a) / 2
        for jj, j in enumerate(range(blk.c0 + 1, blk.c1 + 1)):
            tj = [mpmath.mpf(float(t[j + s])) for s in (-1, 0, 1)]
            for nu in range(k):
                e = 1 - mpmath.mpf(alpha) - nu
                c_nu = mpmath.mpf(1)
                for l in range(1, nu + 1):
                    c_nu *= (1 - mpmath.mpf(alpha) - l) / l
                mi = [(tc - v) ** e for v in tj]
                ref = c_nu / e * ((mi[0] - mi[1]) / (tj[1] - tj[0]) - (mi[1] - mi[2]) / (tj[2] - tj[1]))
                ref *= rho ** nu
                assert abs(B[jj, nu] - float(ref)) <= 1e-12 * abs(float(ref)) + 1e-300


@pytest.mark.parametrize("k", [3, 6, 10, 16])
@pytest.mark.parametrize("alpha,gamma", [(0.3, 1.7 / 0.3), (0.5, 1.0), (0.8, 1.5)])
def test_theorem31_bound(alpha, gamma, k):
    M, leaf = 256, 16
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    for blk in hmatrix.block_tree(t, leaf):
        if blk.kind != "rk":
            continue
        A, B = hmatrix.rk_factors(t, alpha, blk, k)
        err = np.abs(R[blk.r0:blk.r1, blk.c0:blk.c1] - A @ B.T)
        bound = hmatrix.theorem31_bound(t, alpha, blk, k)
        # + a few ulps of the entries themselves
        assert np.all(err <= bound + 1e-13 * np.abs(R[blk.r0:blk.r1, blk.c0:blk.c1])), blk


def test_taylor_error_decays_like_3_to_minus_k():
    M, leaf, alpha = 512, 32, 0.4
    t = l1.graded_mesh(1.0, M, 2.5)
    R = l1.l1_matrix(t, alpha)
    errs = []
    for k in (4, 8, 12):
        Rt, _ = hmatrix.approximate(t, alpha, R, leaf, k)
        errs.append(np.abs(Rt - R).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[0] < 3.0 ** -3 and errs[2] / errs[1] < 3.0 ** -3


# ---------------------------------------------------------------- multigrid (Algorithm 2)

def test_smoother_zeroes_residual_on_last_colour():
    """Gauss-Seidel property: after a sweep the defect vanishes on the colour updated last."""
    for dim, N in ((1, 15), (2, 7)):
        t, h, F = _manufactured(dim, N, 16, 0.5, 2.0)
        R = l1.l1_matrix(t, 0.5)
        rng = np.random.default_rng(0)
        u = wrmg.smooth(R, F, rng.standard_normal(F.shape), h)
        r = wrmg.defect(R, F, u, h)
        last = (wrmg._colour_masks_1d(N) if dim == 1 else wrmg._colour_masks_2d(N))[1]
        assert np.abs(r[:, last]).max() <= 1e-10 * np.abs(F).max()
        assert np.abs(r[:, ~last]).max() > 1e-6


def test_transfer_operators_on_linear_functions():
    """Linear interpolation reproduces linear functions that vanish on the boundary piecewise;
    full weighting of a linear function equals its coarse values."""
    Nc = 7
    xc = np.arange(1, Nc + 1) / (Nc + 1)
    ef = wrmg.prolong((xc * (1 - 0 * xc))[None, :])
    xf = np.arange(1, 2 * Nc + 2) / (2 * Nc + 2)
    assert np.allclose(ef[0, :-1], xf[:-1])     # the last fine point sees the zero boundary
    lin = np.arange(1, 16)[None, :].astype(float)
    assert np.allclose(wrmg.restrict_fw(lin)[0], np.arange(2, 15, 2))
    ec2 = np.outer(xc, xc)[None]
    ef2 = wrmg.prolong(ec2)
    assert np.allclose(ef2[0, :-1, :-1], np.outer(xf[:-1], xf[:-1]))
    lin2 = np.add.outer(np.arange(1, 16), 2 * np.arange(1, 16))[None].astype(float)
    assert np.allclose(wrmg.restrict_fw(lin2)[0], lin2[0][1::2, 1::2])


@pytest.mark.parametrize("dim,N,M", [(1, 31, 32), (2, 15, 16)])
def test_multigrid_converges_to_direct_solution(dim, N, M):
    t, h, F = _manufactured(dim, N, M, 0.5, 2.0)
    R = l1.l1_matrix(t, 0.5)
    u, k, hist = wrmg.solve(R, F, h, 1, 1, 1e-12)
    ud = direct.solve_o1(R, F, h)
    assert k < 15
    assert np.abs(u - ud).max() <= 1e-10 * np.abs(ud).max()


@pytest.mark.parametrize("dim,N,M", [(1, 7, 12), (1, 15, 8), (2, 3, 10), (2, 7, 4)])
def test_direct_level_solve_matches_brute_force(dim, N, M):
    # the sine-transform + per-mode triangular solve against the dense Kronecker system
    t = l1.graded_mesh(1.0, M, 1.7)
    R = l1.l1_matrix(t, 0.4)
    h = 1.0 / (N + 1)
    F = np.random.default_rng(5).standard_normal((M,) + (N,) * dim)
    u = wrmg.direct_level_solve(R, F, h)
    u3 = direct.solve_o3(R, F, h)
    assert np.abs(u - u3).max() <= 1e-12 * np.abs(u3).max()


def test_direct_level_solve_on_one_point_is_the_coarsest_solve():
    t = l1.graded_mesh(1.0, 16, 2.0)
    R = l1.l1_matrix(t, 0.5)
    F = np.random.default_rng(6).standard_normal((16, 1))
    a = wrmg.direct_level_solve(R, F, 0.5)
    b = wrmg.coarsest_solve(R, F, 0.5)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("dim,N,M", [(1, 63, 32), (2, 15, 16)])
def test_exact_coarse_correction_converges_no_slower(dim, N, M):
    # n_direct = 1 is the paper's cycle; an exact coarse-grid correction on the 7-point (1D) or
    # 3x3 (2D) grid reaches the direct solution in no more cycles
    t, h, F = _manufactured(dim, N, M, 0.5, 2.0)
    R = l1.l1_matrix(t, 0.5)
    ud = direct.solve_o1(R, F, h)
    u1, k1, _ = wrmg.solve(R, F, h, 1, 1, 1e-11)
    u7, k7, _ = wrmg.solve(R, F, h, 1, 1, 1e-11, n_direct=7 if dim == 1 else 3)
    assert k7 <= k1
    assert np.abs(u7 - ud).max() <= 1e-9 * np.abs(ud).max()
    # a two-grid cycle with the exact coarse solve equals the full recursion once every
    # coarser level is solved exactly: n_direct = N // 2 is a two-grid method
    v0 = np.random.default_rng(7).standard_normal(F.shape)
    a = wrmg.cycle(R, F, v0, h, 1, 1, n_direct=(N - 1) // 2)
    v = wrmg.smooth(R, F, v0, h)
    ec = direct.solve_o3(R, wrmg.restrict_fw(wrmg.defect(R, F, v, h)), 2.0 * h)
    b = wrmg.smooth(R, F, v + wrmg.prolong(ec), h)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()


def _asymptotic_factor(R, h, N, M, nu, gamma_c, seed=0, ncyc=12):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((M, N))
    F = np.zeros((M, N))
    rs = [np.abs(wrmg.defect(R, F, u, h)).max()]
    for _ in range(ncyc):
        u = wrmg.cycle(R, F, u, h, nu[0], nu[1], gamma_c)
        rs.append(np.abs(wrmg.defect(R, F, u, h)).max())
    return (rs[-1] / rs[-5]) ** 0.25


def test_table2_wcycle_factors():
    for delta, grid, sama, measured in load_golden("table2_factors.txt"):
        if grid != 64:
            continue
        M = int(grid)
        N = M - 1
        t = l1.graded_mesh(1.0, M, (2 - delta) / delta)
        R = l1.l1_matrix(t, delta)
        rho = _asymptotic_factor(R, math.pi / (N + 1), N, M, (0, 1), 2)
        assert abs(rho - measured) <= 0.1 * measured + 0.003, (delta, rho, measured)


def test_table3_vcycle_counts():
    for delta, grid, cycles, factor in load_golden("table3_vcycles_1d.txt"):
        if grid != 128:
            continue
        M = int(grid)
        N = M - 1
        t = l1.graded_mesh(1.0, M, (2 - delta) / delta)
        R = l1.l1_matrix(t, delta)
        u0 = np.random.default_rng(1).standard_normal((M, N))
        _, k, hist = wrmg.solve(R, np.zeros((M, N)), math.pi / (N + 1), 0, 1, 1e-10, u0=u0)
        assert abs(k - cycles) <= 1, (delta, k, cycles)


def test_table5_vcycle_counts_2d():
    for delta, grid, cycles, factor in load_golden("table5_vcycles_2d.txt"):
        if grid != 32:
            continue
        M = int(grid)
        N = M - 1
        t = l1.graded_mesh(1.0, M, (2 - delta) / delta)
        R = l1.l1_matrix(t, delta)
        h = math.pi / (N + 1)
        x = np.arange(1, N + 1) * h
        tt = t[1:]
        S = np.sin(x)[:, None] * np.sin(x)[None, :]
        amp = 2 * (tt ** 3 + tt ** delta) + math.gamma(delta + 1) + math.gamma(4) / math.gamma(4 - delta) * tt ** (3 - delta)
        F = amp[:, None, None] * S[None]
        _, k, _ = wrmg.solve(R, F, h, 1, 1, 1e-10)
        assert abs(k - cycles) <= 1, (delta, k, cycles)
