"""The paper's experiments of Section 5 reproduced through the library on the GPU, and the W-cycle
option (cycle index 2, Algorithm 2's number of coarse-grid cycles) against the oracle.

* W(1,1) and W(0,1) cycles element by element against the oracle's cycle with gamma_c = 2;
* Table 2: multilevel W-cycle factors with one smoothing step (within 10 % + 0.003, as the
  oracle's own pin), at the three printed grids;
* Tables 3 and 4: V(0,1) cycle counts to a 1e-10 residual reduction (1D, random initial guess,
  zero source), every printed grid up to 2048 x 2048 and every printed rank k at 512 x 512 (+-1);
* Tables 5 and 6: V(1,1) cycle counts (2D, u = (t^3 + t^delta) sin x sin y) up to 256^3 and for
  every printed rank at 64^3 (+-1);
* Table 1: the L1 scheme's maximum error for u = E_delta(-t^delta) sin x (f = 0, g = sin x on
  (0, pi)) through the GPU solve with initial data, within 8 % of the printed values, and the
  observed orders log2(E_M / E_2M).
The H-matrix is the paper's form (rank k = 20 Taylor terms) unless a table varies k.  Grids
"N x M" are read as N = M - 1 interior points (N + 1 = 2^L subintervals) on (0, pi).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import hmatrix, l1, wrmg  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402
from tests.conftest import load_golden  # noqa: E402

DEV = "cuda"


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("nu", [(1, 1), (0, 1)])
@pytest.mark.parametrize("dim,N,M,rank", [(1, 63, 64, 0), (1, 127, 128, 12), (2, 15, 64, 10)])
def test_wcycle_matches_oracle(dim, N, M, rank, nu):
    alpha, gamma = 0.4, 2.5
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    Rt = hmatrix.approximate(t, alpha, R, 64, rank)[0] if rank else R
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, rank, 0.0)
    P = fh.Problem(H, dim, N, 1.0)
    P.set_cycle_index(2)
    shape = (M,) + (N,) * dim
    F = inputs.random_field(3, shape)
    u0 = inputs.random_field(4, shape)
    u = dev(u0)
    P.vcycle(u, dev(F), None, *nu)
    ref = wrmg.cycle(Rt, F, u0, 1.0 / (N + 1), nu[0], nu[1], gamma_c=2)
    err = float(np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max())
    assert err < 1e-11, err


def test_cycle_index_changes_the_cycle():
    """A W-cycle is not a V-cycle: the two differ on a 3-level grid, and cycle index 1 restores V."""
    H = fh.HMatrix(0.5, 2.0, 1.0, 64, 64, 0, 0.0)
    P = fh.Problem(H, 1, 15)
    F = dev(inputs.random_field(1, (64, 15)))
    outs = []
    for ci in (1, 2, 1):
        P.set_cycle_index(ci)
        u = torch.zeros_like(F)
        P.vcycle(u, F, None, 1, 1)
        outs.append(u)
    assert float((outs[0] - outs[1]).abs().max()) > 1e-8
    assert float((outs[0] - outs[2]).abs().max()) == 0.0
    with pytest.raises(fh.FhmgError):
        P.set_cycle_index(0)


def _problem(delta, M, N, dim, rank=20):
    gamma = (2 - delta) / delta
    H = fh.HMatrix(delta, gamma, 1.0, M, 64, rank, 0.0)
    return H, fh.Problem(H, dim, N, math.pi)


@pytest.mark.parametrize("grid", [64, 128, 256])
def test_table2_wcycle_factors(grid):
    for delta, g, sama, measured in load_golden("table2_factors.txt"):
        if g != grid:
            continue
        M, N = grid, grid - 1
        H, P = _problem(delta, M, N, 1)
        P.set_cycle_index(2)
        u = dev(np.random.default_rng(0).standard_normal((M, N)))
        F = torch.zeros_like(u)
        rs = [P.residual_norm(u, F)]
        for _ in range(12):
            P.vcycle(u, F, None, 0, 1)
            rs.append(P.residual_norm(u, F))
        rho = (rs[-1] / rs[-5]) ** 0.25
        assert abs(rho - measured) <= 0.1 * measured + 0.003, (delta, grid, rho, measured)


def _vcycles_1d(delta, M, N, rank):
    H, P = _problem(delta, M, N, 1, rank)
    u = dev(np.random.default_rng(1).standard_normal((M, N)))
    k, rr = P.solve(u, torch.zeros_like(u), None, 0, 1, 1e-10, 40)
    return k


@pytest.mark.parametrize("grid", [128, 256, 512, 1024, 2048])
def test_table3_vcycle_counts(grid):
    for delta, g, cycles, factor in load_golden("table3_vcycles_1d.txt"):
        if g == grid:
            k = _vcycles_1d(delta, grid, grid - 1, 20)
            assert abs(k - cycles) <= 1, (delta, grid, k, cycles)


def test_table4_rank_independence():
    for delta, k_rank, cycles, factor in load_golden("table4_vcycles_rank_1d.txt"):
        k = _vcycles_1d(delta, 512, 511, int(k_rank))
        assert abs(k - cycles) <= 1, (delta, k_rank, k, cycles)


def _vcycles_2d(delta, M, N, rank):
    H, P = _problem(delta, M, N, 2, rank)
    t, _ = H.mesh()
    h = math.pi / (N + 1)
    x = np.arange(1, N + 1) * h
    tt = t[1:]
    S = np.sin(x)[:, None] * np.sin(x)[None, :]
    amp = 2 * (tt ** 3 + tt ** delta) + math.gamma(delta + 1) + math.gamma(4) / math.gamma(4 - delta) * tt ** (3 - delta)
    F = dev(amp)[:, None, None] * dev(S)[None]
    u = torch.zeros_like(F)
    k, rr = P.solve(u, F, None, 1, 1, 1e-10, 40)
    return k


@pytest.mark.parametrize("grid", [32, 64])
def test_table5_vcycle_counts_2d(grid):
    for delta, g, cycles, factor in load_golden("table5_vcycles_2d.txt"):
        if g == grid:
            k = _vcycles_2d(delta, grid, grid - 1, 20)
            assert abs(k - cycles) <= 1, (delta, grid, k, cycles)


@pytest.mark.parametrize("grid", [128, 256])
def test_table5_larger_grids(grid):
    """At 128^3 and 256^3 the paper prints 9 cycles, while the run it keeps commented out in its
    source next to the table needed 11-12 at these grids; the method as read here (the oracle's
    Algorithm 2) needs 10-11 at 128^3.  The GPU count equals the oracle's at 128^3 and lies
    within the printed-to-earlier-run band at both grids (the oracle runs the same rank-20 matrix)."""
    for delta, g, cycles, factor in load_golden("table5_vcycles_2d.txt"):
        if g != grid:
            continue
        k = _vcycles_2d(delta, grid, grid - 1, 20)
        assert cycles <= k <= 12, (delta, grid, k)
        if grid == 128:
            M, N = grid, grid - 1
            t = l1.graded_mesh(1.0, M, (2 - delta) / delta)
            Rt = hmatrix.approximate(t, delta, l1.l1_matrix(t, delta), 64, 20)[0]  # the same rank-20 form
            h = math.pi / (N + 1)
            x = np.arange(1, N + 1) * h
            tt = t[1:]
            S = np.sin(x)[:, None] * np.sin(x)[None, :]
            amp = (2 * (tt ** 3 + tt ** delta) + math.gamma(delta + 1)
                   + math.gamma(4) / math.gamma(4 - delta) * tt ** (3 - delta))
            _, k_oracle, _ = wrmg.solve(Rt, amp[:, None, None] * S[None], h, 1, 1, 1e-10)
            assert k == k_oracle, (delta, k, k_oracle)


def test_table6_rank_independence_2d():
    for delta, k_rank, cycles, factor in load_golden("table6_vcycles_rank_2d.txt"):
        k = _vcycles_2d(delta, 64, 63, int(k_rank))
        assert abs(k - cycles) <= 1, (delta, k_rank, k, cycles)


def test_table1_errors_through_gpu_solve():
    """f = 0, g = sin x on (0, pi): the GPU solve with initial data (F = d_{m,m} g) against the
    exact solution E_delta(-t^delta) sin x, N = 1023, the graded mesh r = (2 - delta)/delta."""
    N = 1023
    g = dev(inputs.mittag_leffler_1d(N)[0])
    x = torch.as_tensor(inputs.grid(N, math.pi), device=DEV)
    got = {}
    for delta, M, E_paper in load_golden("table1_errors.txt"):
        M = int(M)
        H, P = _problem(delta, M, N, 1, rank=0)
        t, _ = H.mesh()
        u = torch.zeros((M, N), dtype=torch.float64, device=DEV)
        P.solve(u, torch.zeros_like(u), g, 1, 1, 1e-11, 60, allow_notconv=True)
        exact = dev(l1.mittag_leffler(delta, -t[1:] ** delta))[:, None] * torch.sin(x)[None, :]
        E = float((u - exact).abs().max())
        got[(delta, M)] = E
        assert abs(E - E_paper) <= 0.08 * E_paper, (delta, M, E, E_paper)
    for delta in (0.4, 0.6, 0.8):
        orders = [math.log2(got[(delta, M)] / got[(delta, 2 * M)]) for M in (64, 128, 256)]
        assert all(o > 1.0 for o in orders) and abs(orders[-1] - (2 - delta)) < 0.5, (delta, orders)
