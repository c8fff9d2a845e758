"""The bounded device waits give up cleanly: a test hook (fhmg_problem_inject_timeout) arms the
next walk launch so that every CTA's producer withholds the second chunk of its stream -- a
stage that nothing will ever fill -- and the consumer warps' waits give up after a short poll
limit.  Nothing faults or hangs: the kernel leaves early, every copy it issued lands first, the
call that reads the error word returns FHMG_ETIMEOUT, and the problem stays usable (the next call
gives the same result as a clean run).  One test per walk kernel: the FP64 SIMT walk, the
double-float walk (mixed outer defect) and the tensor-core walk (mixed smoother)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402


def _setup(prec, N, M):
    H = fh.HMatrix(0.5, 2.0, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 1, N, 1.0, prec)
    f = torch.as_tensor(inputs.random_field(1, (M, N)), device="cuda")
    u = torch.as_tensor(inputs.random_field(2, (M, N)), device="cuda")
    return H, P, f, u


@pytest.mark.parametrize("prec", [fh.FP64, fh.MIXED_FP32])
def test_defect_walk_timeout_is_reported_and_cleared(prec):
    H, P, f, u = _setup(prec, 255, 256)
    ref = P.residual_norm(u, f)
    P.inject_timeout(1024)
    with pytest.raises(fh.FhmgError) as e:
        P.residual_norm(u, f)
    assert e.value.status == fh.FHMG_ETIMEOUT
    assert P.residual_norm(u, f) == ref          # the error word was cleared; same result
    torch.cuda.synchronize()                      # the context is intact


def test_tensor_core_smoother_timeout_in_a_solve():
    """Mixed solve on 4095 points (the smoother's 2048-column colours run on the tensor-core walk):
    the armed launch is the first smoother half-sweep; the solve reports FHMG_ETIMEOUT, and a second
    solve from zero equals a clean one."""
    H, P, f, _ = _setup(fh.MIXED_FP32, 4095, 256)
    clean = torch.zeros_like(f)
    k0, _ = P.solve(clean, f, None, 1, 1, 1e-8, 60)
    P.inject_timeout(256)
    u = torch.zeros_like(f)
    with pytest.raises(fh.FhmgError) as e:
        P.solve(u, f, None, 1, 1, 1e-8, 60)
    assert e.value.status == fh.FHMG_ETIMEOUT
    u.zero_()
    k1, _ = P.solve(u, f, None, 1, 1, 1e-8, 60)
    assert k1 == k0 and float((u - clean).abs().max()) == 0.0


def test_inject_rejects_bad_limits():
    H, P, f, u = _setup(fh.FP64, 63, 128)
    for bad in (0, -5, 1 << 30):
        with pytest.raises(fh.FhmgError):
            P.inject_timeout(bad)
