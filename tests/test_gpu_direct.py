"""GPU parity of the exact coarse-level solve (fhmg_problem_set_coarse_direct) against the
oracle's cycle with the same coarse-grid correction (wrmg.cycle(..., n_direct)), and full
solves with it against the per-mode oracle, FP64 and mixed precision.

Tolerances (relative max-norm): one cycle with the same time matrix on both sides 1e-11;
solutions with the recompressed H-matrix (tol 1e-10) 1e-8 (FP64) and 1e-7 (mixed), as for the
plain cycle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, hmatrix, l1, wrmg  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402

DEV = "cuda"

# (alpha, gamma, M, leaf, rank, tol): dense R, the paper's Taylor form of R~
MODES = [
    (0.5, 2.0, 64, 64, 0, 0.0),
    (0.3, 1.7 / 0.3, 256, 32, 12, 0.0),
]


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(x):
    torch.cuda.synchronize()
    return x.cpu().numpy()


def time_matrix(alpha, gamma, M, leaf, rank, tol):
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    if rank > 0:
        R, _ = hmatrix.approximate(t, alpha, R, min(leaf, M), rank)
    return R


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dim,N,nc", [(1, 63, 7), (1, 127, 31), (1, 31, 15), (2, 15, 3), (2, 31, 7)])
def test_vcycle_with_exact_coarse_level(mode, dim, N, nc):
    Rt = time_matrix(*mode)
    M = mode[2]
    H = fh.HMatrix(*mode[:2], 1.0, M, *mode[3:])
    P = fh.Problem(H, dim, N)
    P.set_coarse_direct(nc)
    shape = (M, N) if dim == 1 else (M, N, N)
    u0 = inputs.random_field(21, shape)
    F = inputs.random_field(22, shape) * 10
    u = dev(u0)
    P.vcycle(u, dev(F), None, 1, 1)
    ref = wrmg.cycle(Rt, F, u0, 1.0 / (N + 1), 1, 1, n_direct=nc)
    assert rel(host(u), ref) < 1e-11


def test_switching_back_restores_the_paper_cycle():
    mode = MODES[0]
    M, N = mode[2], 63
    H = fh.HMatrix(*mode[:2], 1.0, M, *mode[3:])
    u0 = inputs.random_field(23, (M, N))
    F = dev(inputs.random_field(24, (M, N)))
    P = fh.Problem(H, 1, N)
    a = dev(u0)
    P.vcycle(a, F, None, 1, 1)
    P.set_coarse_direct(15)
    P.set_coarse_direct(1)
    b = dev(u0)
    P.vcycle(b, F, None, 1, 1)
    assert torch.equal(a, b)


def test_invalid_sizes_are_rejected():
    H = fh.HMatrix(0.5, 2.0, 1.0, 64, 64, 0, 0.0)
    P = fh.Problem(H, 1, 63)
    for bad in (-1, 5, 63, 127):
        with pytest.raises(fh.FhmgError):
            P.set_coarse_direct(bad)
    P.set_coarse_direct(0)
    P.set_coarse_direct(31)


def _mode_solution(alpha, gamma, M, N, dim):
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    h = 1.0 / (N + 1)
    lam = dim * 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    a, s = inputs.manufactured(t[1:], N, dim, alpha)
    return a, s, direct.solve_o2_mode(R, lam, a)


@pytest.mark.parametrize("prec", [fh.FP64, fh.MIXED_FP32])
@pytest.mark.parametrize("nc", [63, 255])
def test_full_size_1d_with_exact_coarse_level(prec, nc):
    """N=4095, M=4096, alpha=.5, H tol 1e-10: every entry against the per-mode oracle, and no more
    cycles than the paper's recursion needs."""
    alpha, gamma, M, N = 0.5, 3.0, 4096, 4095
    a, s, w = _mode_solution(alpha, gamma, M, N, 1)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    f = dev(a)[:, None] * dev(s)[None, :]
    ref = torch.as_tensor(w, device=DEV)[:, None] * dev(s)[None, :]
    ks = []
    for direct_n in (1, nc):
        P = fh.Problem(H, 1, N, prec=prec)
        P.set_coarse_direct(direct_n)
        u = torch.zeros((M, N), dtype=torch.float64, device=DEV)
        k, rr = P.solve(u, f, None, 1, 1, 1e-8, 30)
        assert rr <= 1e-8
        err = float((u - ref).abs().max() / ref.abs().max())
        assert err < (1e-8 if prec == fh.FP64 else 1e-7), (direct_n, err, k, rr)
        ks.append(k)
    assert ks[1] <= ks[0]


@pytest.mark.parametrize("prec", [fh.FP64, fh.MIXED_FP32])
def test_full_size_2d_with_exact_coarse_level(prec):
    """2D N=511^2, M=1024, alpha=.4, gamma=2.5 with the 15 x 15 level solved exactly."""
    alpha, gamma, M, N = 0.4, 2.5, 1024, 511
    a, s, w = _mode_solution(alpha, gamma, M, N, 2)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 2, N, prec=prec)
    P.set_coarse_direct(15)
    s2 = dev(s)  # already the 2D product of sines
    f = dev(a)[:, None, None] * s2[None]
    u = torch.zeros((M, N, N), dtype=torch.float64, device=DEV)
    k, rr = P.solve(u, f, None, 1, 1, 1e-8, 30)
    assert rr <= 1e-8
    ref = torch.as_tensor(w, device=DEV)[:, None, None] * s2[None]
    err = float((u - ref).abs().max() / ref.abs().max())
    assert err < (1e-8 if prec == fh.FP64 else 1e-7), (err, k, rr)
