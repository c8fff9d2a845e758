"""fhmg_residual_norm_noalloc (through the C-ABI) against fhmg_residual_norm.

The allocation-free entry point serves callers that cannot allocate device memory while their
solve loop runs; it keeps its scratch in a fixed library-owned device array.  Two calls in a row
with different iterates must both match the allocating entry point: the second call sees a
smaller defect, so a stale max-norm accumulator from the first call would show up.
This file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402


@pytest.mark.parametrize("dim,N,M,leaf,tol", [(1, 63, 64, 64, 0.0), (1, 1023, 512, 64, 1e-10), (2, 31, 256, 32, 1e-10)])
def test_noalloc_norm_matches_allocating_entry_point(dim, N, M, leaf, tol):
    H = fh.HMatrix(0.5, 2.0, 1.0, M, leaf, 0, tol)
    P = fh.Problem(H, dim, N)
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


def test_noalloc_rejects_oversized_problem():
    H = fh.HMatrix(0.5, 2.0, 1.0, 4096, 64, 0, 1e-10)
    P = fh.Problem(H, 1, 1023)
    f = torch.zeros((4096, 1023), dtype=torch.float64, device="cuda")
    with pytest.raises(fh.FhmgError) as e:
        P.residual_norm_noalloc(f, f)
    assert e.value.status == fh.FHMG_EINVAL
