"""The library's two-grid mode-analysis predictor (fhmg_sama_two_grid, host code) against the
oracle's (independent numpy restatement, itself pinned by the assembled two-grid operator) and
against Table 2's SAMA column (Section 5)."""
import math

import pytest

import paper_1706_07632_gb300 as fh
from oracle import l1, sama
from tests.conftest import load_golden


@pytest.mark.parametrize("nu", [(0, 1), (1, 1), (2, 1)])
@pytest.mark.parametrize("dim,N,M,alpha,Lx", [(1, 63, 64, 0.3, math.pi), (1, 127, 128, 0.6, 1.0), (2, 15, 32, 0.5, 1.0),
                                              (2, 31, 64, 0.4, math.pi)])
def test_library_predictor_matches_oracle(dim, N, M, alpha, Lx, nu):
    gamma = (2 - alpha) / alpha
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 0.0)
    t = l1.graded_mesh(1.0, M, gamma)
    ref = sama.two_grid_factor(l1.l1_matrix(t, alpha), dim, N, Lx / (N + 1), *nu)
    got = H.sama_two_grid(dim, N, Lx, *nu)
    assert abs(got - ref) <= 1e-9 * max(ref, 1e-3), (got, ref)


def test_library_predictor_table2():
    for delta, grid, sama_p, measured in load_golden("table2_factors.txt"):
        M = int(grid)
        H = fh.HMatrix(delta, (2 - delta) / delta, 1.0, M, 64, 20, 0.0)
        rho = H.sama_two_grid(1, M - 1, math.pi, 0, 1)
        assert abs(rho - sama_p) <= 0.003, (delta, grid, rho, sama_p)


def test_predictor_rejects_bad_arguments():
    H = fh.HMatrix(0.5, 2.0, 1.0, 64, 64, 0, 0.0)
    for args in [(3, 15, 1.0, 0, 1), (1, 16, 1.0, 0, 1), (1, 15, 1.0, 0, 0), (1, 1, 1.0, 0, 1)]:
        with pytest.raises(fh.FhmgError):
            H.sama_two_grid(*args)
