"""GPU parity: every hot-path step through the C-ABI against the oracle, element by element,
on seeded inputs spanning several column tiles and a ragged tail; full solves against the
direct oracle; full-size configurations against the per-mode oracle.

Tolerances (relative max-norm):
* same time matrix on both sides (dense R, or the paper's Taylor form of R~ with k terms):
  1e-11 for single steps and cycles (double rounding of O(M) sums);
* solutions with dense R: 1e-10; with the recompressed H-matrix (tol 1e-10): 1e-8.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, hmatrix, l1, wrmg  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402

DEV = "cuda"


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(x):
    torch.cuda.synchronize()
    return x.cpu().numpy()


_cache = {}


def oracle_R(alpha, gamma, M):
    key = ("R", alpha, gamma, M)
    if key not in _cache:
        t = l1.graded_mesh(1.0, M, gamma)
        _cache[key] = (t, l1.l1_matrix(t, alpha))
    return _cache[key]


def oracle_time_matrix(alpha, gamma, M, leaf, rank, tol):
    """The time matrix the oracle pairs with a library mode: dense R, or the paper's Taylor R~."""
    t, R = oracle_R(alpha, gamma, M)
    if rank > 0:
        Rt, _ = hmatrix.approximate(t, alpha, R, min(leaf, M), rank)
        return t, Rt
    return t, R


# (alpha, gamma, M, leaf, rank, tol): dense, paper Taylor form, recompressed
MODES = [
    (0.5, 2.0, 64, 64, 0, 0.0),
    (0.3, 1.7 / 0.3, 256, 32, 12, 0.0),
    (0.8, 1.5, 512, 64, 10, 0.0),
    (0.4, 2.5, 128, 16, 14, 0.0),
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("ncols", [1, 37, 1029])
def test_line_solve_alg4(mode, ncols):
    alpha, gamma, M, leaf, rank, tol = mode
    t, Rt = oracle_time_matrix(*mode)
    H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, rank, tol)
    P = fh.Problem(H, 1, 63)
    B = inputs.random_field(ncols, (M, ncols))
    X = torch.empty((M, ncols), dtype=torch.float64, device=DEV)
    for level in (0, 3, 5):
        h = 1.0 / (2 ** (level + 1))
        P.line_solve(level, X, dev(B))
        ref = direct.solve_o2_mode(Rt, 2.0 / h ** 2, B)
        assert rel(host(X), ref) < 1e-11
    # in place
    Xb = dev(B)
    P.line_solve(5, Xb, Xb)
    assert rel(host(Xb), direct.solve_o2_mode(Rt, 2.0 * 64 ** 2, B)) < 1e-11


@pytest.mark.parametrize("mode", MODES)
def test_hmatvec_alg3(mode):
    alpha, gamma, M, leaf, rank, tol = mode
    t, Rt = oracle_time_matrix(*mode)
    H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, rank, tol)
    P = fh.Problem(H, 1, 15)
    X = inputs.random_field(7, (M, 301))
    Y = torch.empty_like(dev(X))
    P.hmatvec(Y, dev(X))
    assert rel(host(Y), Rt @ X) < 1e-11


def _level_problem(mode, dim, N):
    alpha, gamma, M, leaf, rank, tol = mode
    H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, rank, tol)
    return H, fh.Problem(H, dim, N)


@pytest.mark.parametrize("mode", MODES[:3])
@pytest.mark.parametrize("dim,N", [(1, 63), (1, 255), (2, 15), (2, 31)])
def test_smoother_halfsweeps(mode, dim, N):
    t, Rt = oracle_time_matrix(*mode)
    M = mode[2]
    H, P = _level_problem(mode, dim, N)
    shape = (M, N) if dim == 1 else (M, N, N)
    u0 = inputs.random_field(1, shape)
    F = inputs.random_field(2, shape) * 100
    u = dev(u0)
    P.smooth(u, dev(F), 2)
    h = 1.0 / (N + 1)
    ref = wrmg.smooth(Rt, F, wrmg.smooth(Rt, F, u0, h), h)
    assert rel(host(u), ref) < 1e-11


@pytest.mark.parametrize("mode", MODES[:3])
@pytest.mark.parametrize("dim,N", [(1, 127), (2, 31)])
def test_residual_restriction_prolongation(mode, dim, N):
    t, Rt = oracle_time_matrix(*mode)
    alpha, M = mode[0], mode[2]
    H, P = _level_problem(mode, dim, N)
    shape = (M, N) if dim == 1 else (M, N, N)
    u0 = inputs.random_field(3, shape)
    f = inputs.random_field(4, shape)
    g = inputs.random_field(5, shape[1:])
    h = 1.0 / (N + 1)
    F = direct.rhs_with_initial(f, l1.initial_coeff(t, alpha), g)
    # full defect with initial data
    r = torch.empty_like(dev(u0))
    P.residual(dev(u0), dev(f), dev(g), r)
    ref = wrmg.defect(Rt, F, u0, h)
    assert rel(host(r), ref) < 1e-11
    # restricted defect (time operator commuted with full weighting)
    Nc = (N - 1) // 2
    cshape = (M, Nc) if dim == 1 else (M, Nc, Nc)
    rc = torch.empty(cshape, dtype=torch.float64, device=DEV)
    P.restrict_residual(dev(u0), dev(F), rc)
    assert rel(host(rc), wrmg.restrict_fw(ref)) < 1e-11
    # prolongation + correction
    e = inputs.random_field(6, cshape)
    u = dev(u0)
    P.prolong_correct(u, dev(e))
    assert rel(host(u), u0 + wrmg.prolong(e)) < 1e-14


@pytest.mark.parametrize("mode", MODES[:3])
@pytest.mark.parametrize("dim,N,nu", [(1, 63, (1, 1)), (1, 127, (0, 1)), (2, 15, (1, 1)), (2, 31, (1, 2))])
def test_vcycle_matches_algorithm2(mode, dim, N, nu):
    t, Rt = oracle_time_matrix(*mode)
    M = mode[2]
    H, P = _level_problem(mode, dim, N)
    shape = (M, N) if dim == 1 else (M, N, N)
    u0 = inputs.random_field(8, shape)
    F = inputs.random_field(9, shape) * 10
    u = dev(u0)
    P.vcycle(u, dev(F), None, *nu)
    ref = wrmg.cycle(Rt, F, u0, 1.0 / (N + 1), *nu)
    assert rel(host(u), ref) < 1e-11


def test_coarsest_single_point():
    mode = MODES[0]
    t, Rt = oracle_time_matrix(*mode)
    for dim in (1, 2):
        H, P = _level_problem(mode, dim, 1)
        shape = (64, 1) if dim == 1 else (64, 1, 1)
        F = inputs.random_field(10, shape)
        u = torch.zeros(shape, dtype=torch.float64, device=DEV)
        P.vcycle(u, dev(F), None, 1, 1)
        assert rel(host(u), wrmg.coarsest_solve(Rt, F, 0.5)) < 1e-12


def test_config1_dense_solve():
    """1D, N=63, M=64, alpha=.5, gamma=2, dense R, V(1,1) to 1e-10: GPU vs direct oracle."""
    alpha, gamma, M, N = 0.5, 2.0, 64, 63
    t, R = oracle_R(alpha, gamma, M)
    a, s = inputs.manufactured(t[1:], N, 1, alpha)
    f = np.outer(a, s)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 0.0)
    P = fh.Problem(H, 1, N)
    u = torch.zeros((M, N), dtype=torch.float64, device=DEV)
    k, rr = P.solve(u, dev(f), None, 1, 1, 1e-10, 50)
    ud = direct.solve_o1(R, f, 1.0 / (N + 1))
    assert rel(host(u), ud) < 1e-10
    _, k_or, _ = wrmg.solve(R, f, 1.0 / (N + 1), 1, 1, 1e-10)
    assert k == k_or and rr <= 1e-10


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
def test_config2_hmatrix_solve_small(alpha):
    """1D H-matrix (leaf 64, tol 1e-10) at N=511, M=512 against the direct oracle."""
    gamma = (2 - alpha) / alpha
    M, N = 512, 511
    t, R = oracle_R(alpha, gamma, M)
    a, s = inputs.manufactured(t[1:], N, 1, alpha)
    f = np.outer(a, s) + 0.1 * inputs.random_field(11, (M, N))
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 1, N)
    u = torch.zeros((M, N), dtype=torch.float64, device=DEV)
    # run to the FP64 residual floor (~1e-10 here), then compare the solution
    k, rr = P.solve(u, dev(f), None, 1, 1, 1e-11, 25, allow_notconv=True)
    assert rr < 1e-9
    ud = direct.solve_o1(R, f, 1.0 / (N + 1))
    assert rel(host(u), ud) < 1e-8


def _mode_solution(alpha, gamma, M, N, dim):
    t, R = oracle_R(alpha, gamma, M)
    h = 1.0 / (N + 1)
    lam = dim * 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    a, s = inputs.manufactured(t[1:], N, dim, alpha)
    w = direct.solve_o2_mode(R, lam, a)
    return t, a, s, w


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
def test_config2_full_size(alpha):
    """N=4095, M=4096, H-matrix tol 1e-10, FP64: every entry against the per-mode oracle."""
    gamma = (2 - alpha) / alpha
    M, N = 4096, 4095
    t, a, s, w = _mode_solution(alpha, gamma, M, N, 1)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 1, N)
    f = dev(a)[:, None] * dev(s)[None, :]
    u = torch.zeros((M, N), dtype=torch.float64, device=DEV)
    # the max-norm residual floor of FP64 at h = 1/4096 is ~eps * 4/h^2 * |u| / |f| ~ 6e-9
    k, rr = P.solve(u, f, None, 1, 1, 1e-10, 20, allow_notconv=True)
    assert rr < 1e-8
    ref = torch.as_tensor(w, device=DEV)[:, None] * dev(s)[None, :]
    err = float((u - ref).abs().max() / ref.abs().max())
    assert err < 1e-8, (err, k, rr)


def test_config3_full_size_2d():
    """2D N=511^2, M=1024, alpha=.4, gamma=2.5, H tol 1e-10: every entry vs the per-mode oracle."""
    alpha, gamma, M, N = 0.4, 2.5, 1024, 511
    t, a, s, w = _mode_solution(alpha, gamma, M, N, 2)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 2, N)
    f = dev(a)[:, None, None] * dev(s)[None]
    u = torch.zeros((M, N, N), dtype=torch.float64, device=DEV)
    k, rr = P.solve(u, f, None, 1, 1, 1e-11, 20, allow_notconv=True)
    assert rr < 1e-9
    ref = torch.as_tensor(w, device=DEV)[:, None, None] * dev(s)[None]
    err = float((u - ref).abs().max() / ref.abs().max())
    assert err < 1e-8, (err, k, rr)


def test_initial_data_mittag_leffler():
    """f = 0, g = sin x on (0, pi) (Section 5.1): GPU solve against the per-mode oracle."""
    delta, M, N = 0.6, 128, 127
    gamma = (2 - delta) / delta
    t, R = oracle_R(delta, gamma, M)
    g, Lx = inputs.mittag_leffler_1d(N)
    h = Lx / (N + 1)
    w = direct.solve_o2_mode(R, 4.0 / h ** 2 * math.sin(h / 2) ** 2, l1.initial_coeff(t, delta))
    H = fh.HMatrix(delta, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 1, N, Lx)
    u = torch.zeros((M, N), dtype=torch.float64, device=DEV)
    P.solve(u, torch.zeros((M, N), dtype=torch.float64, device=DEV), dev(g), 0, 1, 1e-10, 60)
    assert rel(host(u), np.outer(w, g)) < 1e-8


def test_cycle_counts_match_oracle_table3_setting():
    """V(0,1) from a random guess, 128 x 128 (Table 3 setting): same cycle count as the oracle."""
    delta, M, N = 0.4, 128, 127
    gamma = (2 - delta) / delta
    t, R = oracle_R(delta, gamma, M)
    H = fh.HMatrix(delta, gamma, 1.0, M, 64, 0, 0.0)
    P = fh.Problem(H, 1, N, math.pi)
    u0 = inputs.random_field(1, (M, N))
    u = dev(u0)
    k, _ = P.solve(u, torch.zeros_like(u), None, 0, 1, 1e-10, 40)
    _, k_or, _ = wrmg.solve(R, np.zeros((M, N)), math.pi / (N + 1), 0, 1, 1e-10, u0=u0)
    assert k == k_or


def test_solve_host_buffers():
    alpha, gamma, M, N = 0.5, 2.0, 64, 63
    t, R = oracle_R(alpha, gamma, M)
    a, s = inputs.manufactured(t[1:], N, 1, alpha)
    f = np.ascontiguousarray(np.outer(a, s))
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 0.0)
    P = fh.Problem(H, 1, N)
    u = np.zeros((M, N))
    P.solve_host(u, f, None, 1, 1, 1e-10, 50)
    assert rel(u, direct.solve_o1(R, f, 1.0 / (N + 1))) < 1e-10


def test_nan_source_is_reported():
    H = fh.HMatrix(0.5, 2.0, 1.0, 64, 64, 0, 0.0)
    P = fh.Problem(H, 1, 15)
    f = torch.zeros((64, 15), dtype=torch.float64, device=DEV)
    f[3, 4] = float("nan")
    u = torch.zeros_like(f)
    with pytest.raises(fh.FhmgError) as e:
        P.solve(u, f, None, 1, 1, 1e-10, 5)
    assert e.value.status == fh.FHMG_ENAN
