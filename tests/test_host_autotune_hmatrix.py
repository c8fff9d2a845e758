"""The host-side H-matrix form tuner (fhmg_autotune_hmatrix, no GPU): the chosen (rank, tol) meets the
error target against the oracle's exact L1 matrix (Section 2), and no candidate of the documented
list that meets it has fewer H-matvec flops (brute force over the list); tighter targets never
cost fewer flops; target 0 gives R itself."""
import numpy as np
import pytest

import paper_1706_07632_gb300 as fh
from oracle import l1

CANDS = [(k, 0.0) for k in (4, 6, 8, 10, 12, 16, 20)] + [(0, t) for t in (1e-6, 1e-8, 1e-10, 1e-12, 1e-14)] + [(0, 0.0)]


def row_rel_err(Rt, R):
    scale = np.abs(R).max(axis=1)
    ok = scale > 0
    return float((np.abs(np.tril(Rt) - np.tril(R)).max(axis=1)[ok] / scale[ok]).max())


@pytest.mark.parametrize("alpha,gamma,M,leaf", [(0.55, 2.0, 512, 64), (0.3, 1.7 / 0.3, 256, 32), (0.8, 1.0, 256, 64)])
@pytest.mark.parametrize("target", [1e-6, 1e-10, 1e-13])
def test_choice_meets_target_and_is_cheapest(alpha, gamma, M, leaf, target):
    r = fh.autotune_hmatrix(alpha, gamma, 1.0, M, leaf, target)
    H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, r["rank"], r["tol"])
    # against the oracle's exact R (the library's own dense R agrees with it to 1e-12 relative)
    t = l1.graded_mesh(1.0, M, gamma)
    Ro = l1.l1_matrix(t, alpha)
    assert row_rel_err(H.dense(), Ro) <= target + 2e-12
    assert H.flops_per_column() == r["flops_per_column"]
    # brute force over the candidate list, errors against the library's exact dense R
    R = fh.HMatrix(alpha, gamma, 1.0, M, leaf, 0, 0.0).dense()
    assert r["err"] == pytest.approx(row_rel_err(H.dense(), R), rel=1e-9, abs=1e-300)
    for k, tol in CANDS:
        C = fh.HMatrix(alpha, gamma, 1.0, M, leaf, k, tol)
        if row_rel_err(C.dense(), R) <= target:
            assert C.flops_per_column() >= r["flops_per_column"]


def test_tighter_targets_cost_no_fewer_flops_and_zero_gives_R():
    fl = [fh.autotune_hmatrix(0.5, 2.0, 1.0, 512, 64, t)["flops_per_column"] for t in (1e-4, 1e-8, 1e-12, 1e-15)]
    assert fl == sorted(fl)
    r = fh.autotune_hmatrix(0.5, 2.0, 1.0, 512, 64, 0.0)
    assert (r["rank"], r["tol"], r["err"]) == (0, 0.0, 0.0)
    assert r["flops_per_column"] == fh.HMatrix(0.5, 2.0, 1.0, 512, 64, 0, 0.0).flops_per_column()


@pytest.mark.parametrize("args", [(0.5, 2.0, 1.0, 512, 64, -1.0), (0.5, 2.0, 1.0, 384, 64, 1e-10),
                                  (1.2, 2.0, 1.0, 512, 64, 1e-10)])
def test_invalid_arguments(args):
    with pytest.raises(fh.FhmgError) as e:
        fh.autotune_hmatrix(*args)
    assert e.value.status == fh.FHMG_EINVAL
