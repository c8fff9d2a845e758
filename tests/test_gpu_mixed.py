"""GPU parity of the mixed-precision path (FP32 H-matrix products inside V-cycles on the
correction equation, FP64 defect / stencil / diagonal; defect correction to the same FP64
residual tolerance as the FP64 path).

The accuracy claim is checked independently: the oracle recomputes the defect of the returned
iterate with its own dense R, and the iterate is compared with the oracle's direct solution.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, l1  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402

DEV = "cuda"


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
@pytest.mark.parametrize("dim,N,M", [(1, 511, 512), (2, 63, 128)])
def test_mixed_reaches_fp64_tolerance(alpha, dim, N, M, storage):
    gamma = (2 - alpha) / alpha
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    a, s = inputs.manufactured(t[1:], N, dim, alpha)
    f = a.reshape((-1,) + (1,) * dim) * s[None] + 0.05 * inputs.random_field(3, (M,) + (N,) * dim)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, dim, N, 1.0, fh.MIXED_FP32)
    P.set_mixed_storage(storage)
    u = torch.zeros(f.shape, dtype=torch.float64, device=DEV)
    k, rr = P.solve(u, dev(f), None, 1, 1, 1e-8, 60)
    assert rr <= 1e-8
    uh = u.cpu().numpy()
    h = 1.0 / (N + 1)
    r = direct.residual(R, f, uh, h)
    assert np.abs(r).max() <= 2e-8 * np.abs(f).max()          # oracle's own defect, dense R
    ud = direct.solve_o1(R, f, h)
    assert np.abs(uh - ud).max() <= 1e-6 * np.abs(ud).max()


def test_mixed_full_size_1d():
    """N=4095, M=4096, alpha=.5 (the benchmark workload) to relres 1e-8, vs the per-mode oracle."""
    alpha, M, N = 0.5, 4096, 4095
    gamma = (2 - alpha) / alpha
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    h = 1.0 / (N + 1)
    a, s = inputs.manufactured(t[1:], N, 1, alpha)
    w = direct.solve_o2_mode(R, 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2, a)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 1, N, 1.0, fh.MIXED_FP32)
    f = dev(a)[:, None] * dev(s)[None, :]
    u = torch.zeros_like(f)
    k, rr = P.solve(u, f, None, 1, 1, 1e-8, 60)
    ref = dev(w)[:, None] * dev(s)[None, :]
    err = float((u - ref).abs().max() / ref.abs().max())
    assert rr <= 1e-8 and err < 1e-7, (k, rr, err)


def test_mixed_full_size_2d():
    """N=511^2, M=1024, alpha=.4, gamma=2.5 (the 2D workload) to relres 1e-8, vs the per-mode oracle."""
    alpha, gamma, M, N = 0.4, 2.5, 1024, 511
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    h = 1.0 / (N + 1)
    a, s = inputs.manufactured(t[1:], N, 2, alpha)
    w = direct.solve_o2_mode(R, 8.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2, a)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 2, N, 1.0, fh.MIXED_FP32)
    f = dev(a)[:, None, None] * dev(s)[None]
    u = torch.zeros_like(f)
    k, rr = P.solve(u, f, None, 1, 1, 1e-8, 60)
    ref = dev(w)[:, None, None] * dev(s)[None]
    err = float((u - ref).abs().max() / ref.abs().max())
    assert rr <= 1e-8 and err < 1e-7, (k, rr, err)
