"""fhmg_residual_norm_noalloc (through the C-ABI) against fhmg_residual_norm and the oracle.

The allocation-free entry point serves callers that cannot allocate device memory while their
solve loop runs; it keeps its scratch in a fixed library-owned device array.  Two calls in a row
with different iterates must both match the allocating entry point (within 1e-12 relative): the
second call sees a smaller defect, so a stale max-norm accumulator from the first call would show
up.  Where the oracle holds the same time matrix (dense R, or the paper's Taylor form), the norm is
also checked against the oracle's own defect (1e-11 relative).
This file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, hmatrix, l1  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402


@pytest.mark.parametrize("prec", [fh.FP64, fh.MIXED_FP32])
@pytest.mark.parametrize("dim,N,M,leaf,tol", [(1, 63, 64, 64, 0.0), (1, 1023, 512, 64, 1e-10), (2, 31, 256, 32, 1e-10)])
def test_noalloc_norm_matches_allocating_entry_point(dim, N, M, leaf, tol, prec):
    H = fh.HMatrix(0.5, 2.0, 1.0, M, leaf, 0, tol)
    P = fh.Problem(H, dim, N, 1.0, prec)
    shape = (M,) + (N,) * dim
    f = torch.as_tensor(inputs.random_field(1, shape), device="cuda")
    u1 = torch.as_tensor(inputs.random_field(2, shape), device="cuda")
    u2 = torch.zeros_like(u1)
    P.solve(u2, f, None, 1, 1, 1e-6, 30, allow_notconv=True)     # an iterate with a much smaller defect
    for u in (u1, u2):
        ref = P.residual_norm(u, f)
        got = P.residual_norm_noalloc(u, f)
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)
    assert P.residual_norm(u2, f) < 1e-3 * P.residual_norm(u1, f)


@pytest.mark.parametrize("prec", [fh.FP64, fh.MIXED_FP32])
@pytest.mark.parametrize("dim,N,M,leaf,rank", [(1, 127, 256, 64, 0), (1, 255, 512, 64, 14), (2, 31, 128, 32, 12)])
def test_noalloc_norm_matches_oracle_defect(dim, N, M, leaf, rank, prec):
    """Same time matrix on both sides (dense R for rank 0, the paper's Taylor form otherwise):
    the allocation-free max-norm equals the oracle's max |F - A u| on two iterates in a row."""
    alpha, gamma = 0.6, 1.8
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    Rt = hmatrix.approximate(t, alpha, R, leaf, rank)[0] if rank else R
    H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, rank, 0.0)
    P = fh.Problem(H, dim, N, 1.0, prec)
    shape = (M,) + (N,) * dim
    f = inputs.random_field(7, shape)
    h = 1.0 / (N + 1)
    for seed, scale in ((8, 1.0), (9, 1e-3)):
        u = inputs.random_field(seed, shape) * scale
        got = P.residual_norm_noalloc(torch.as_tensor(u, device="cuda"), torch.as_tensor(f, device="cuda"))
        ref = float(np.abs(direct.residual(Rt, f, u, h)).max())
        assert abs(got - ref) <= 1e-11 * ref, (got, ref)


def test_noalloc_rejects_oversized_problem():
    H = fh.HMatrix(0.5, 2.0, 1.0, 4096, 64, 0, 1e-10)
    P = fh.Problem(H, 1, 1023)
    f = torch.zeros((4096, 1023), dtype=torch.float64, device="cuda")
    with pytest.raises(fh.FhmgError) as e:
        P.residual_norm_noalloc(f, f)
    assert e.value.status == fh.FHMG_EINVAL
