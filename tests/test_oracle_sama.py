"""Pins of the oracle's two-grid mode analysis (Section 5, Table 2).

The brute-force check does not eigen-solve the assembled operator (it is far from normal, so the
eigenvalues of the full matrix are ill-conditioned); it checks the structure the analysis rests on
and the matrices it uses: the two-grid operator, assembled column by column from Algorithm 2's
pieces and transformed to the orthonormal sine basis in space, (i) couples each sine mode only with
its partners under k -> N+1-k (pairs in 1D, quadruples in 2D), (ii) is block lower triangular in
time within each group, and (iii) its time-diagonal blocks equal, entry by entry, the per-mode
matrices of the analysis with R replaced by R_mm.  The factor then reproduces Table 2's SAMA column.
"""
import math

import numpy as np
import pytest

from oracle import l1, sama
from tests.conftest import load_golden


def _dst(N):
    n = np.arange(1, N + 1)
    return math.sqrt(2.0 / (N + 1)) * np.sin(np.pi * np.outer(n, n) / (N + 1))  # symmetric, orthogonal


@pytest.mark.parametrize("nu", [(0, 1), (1, 1), (1, 0)])
@pytest.mark.parametrize("dim,N,M,alpha", [(1, 15, 8, 0.4), (1, 31, 4, 0.7), (2, 7, 4, 0.5)])
def test_mode_structure_of_assembled_operator(dim, N, M, alpha, nu):
    t = l1.graded_mesh(1.0, M, (2 - alpha) / alpha)
    R = l1.l1_matrix(t, alpha)
    h = math.pi / (N + 1)
    T = sama.two_grid_operator(R, dim, N, h, *nu)
    Q = _dst(N) if dim == 1 else np.kron(_dst(N), _dst(N))
    nsp = Q.shape[0]
    # index (m, p) -> m * nsp + p; transform space: Tm = (I_M x Q) T (I_M x Q)
    big = np.kron(np.eye(M), Q)
    Tm = (big @ T @ big).reshape(M, nsp, M, nsp)  # [m, mode, m', mode']
    scale = np.abs(Tm).max()
    half = (N - 1) // 2
    for k in range(1, half + 1):
        kp = N + 1 - k
        if dim == 1:
            group = [k - 1, kp - 1]
            cs = (math.cos(k * math.pi / (N + 1)),)
        else:
            for l in range(1, half + 1):
                lp = N + 1 - l
                # ordering of the analysis: (k,l), (k',l'), (k',l), (k,l'); index (l - 1) * N + (k - 1)
                group = [(l - 1) * N + k - 1, (lp - 1) * N + kp - 1, (l - 1) * N + kp - 1, (lp - 1) * N + k - 1]
                _check_group(Tm, group, nsp, M, R, dim, h, nu, scale, (math.cos(k * math.pi / (N + 1)), math.cos(l * math.pi / (N + 1))))
            continue
        _check_group(Tm, group, nsp, M, R, dim, h, nu, scale, cs)


def _check_group(Tm, group, nsp, M, R, dim, h, nu, scale, cs):
    others = [q for q in range(nsp) if q not in group]
    # (i) no coupling from the group to modes outside it
    assert np.abs(Tm[:, others][:, :, :, group]).max() <= 1e-10 * scale
    blk = Tm[:, group][:, :, :, group]  # [m, a, m', b]
    for m in range(M):
        # (ii) lower triangular in time
        if m + 1 < M:
            assert np.abs(blk[m, :, m + 1:, :]).max() <= 1e-10 * scale
        # (iii) the time-diagonal block is the analysis matrix at R_mm
        want = sama._group_1d(R[m, m], cs[0], h, *nu) if dim == 1 else sama._group_2d(R[m, m], cs[0], cs[1], h, *nu)
        got = blk[m, :, m, :]
        assert np.abs(got - want).max() <= 1e-9 * max(1.0, np.abs(want).max()), (m, got, want)


def test_table2_sama_column():
    for delta, grid, sama_p, measured in load_golden("table2_factors.txt"):
        M = int(grid)
        N = M - 1
        t = l1.graded_mesh(1.0, M, (2 - delta) / delta)
        R = l1.l1_matrix(t, delta)
        rho = sama.two_grid_factor(R, 1, N, math.pi / (N + 1), 0, 1)
        assert abs(rho - sama_p) <= 0.003, (delta, grid, rho, sama_p)
