"""The algebraic (adaptive cross approximation) construction of the low-rank blocks, against the
oracle's dense L1 matrix R (Section 2) block by block: each admissible block of the ACA-built R~
deviates from R by at most 2 tol ||R_b||_F in the 2-norm (cross approximation to 0.01 tol, then
truncation at tol * sigma_1 <= tol ||R_b||_F); dense blocks are exact."""
import numpy as np
import pytest

import paper_1706_07632_gb300 as fh
from oracle import hmatrix, l1


@pytest.mark.parametrize("alpha,gamma,M,leaf,tol", [(0.3, 1.7 / 0.3, 2048, 64, 1e-10), (0.5, 3.0, 1024, 64, 1e-10),
                                                    (0.8, 1.5, 256, 32, 1e-8)])
def test_aca_blocks_within_tolerance(alpha, gamma, M, leaf, tol):
    H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, 0, tol, lowrank="aca")
    Rt = H.dense()
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    info = H.info()
    assert info["n_lowrank"] > 0 and info["max_rank"] <= 16
    for b in hmatrix.block_tree(t, leaf):
        if b.kind == "zero":
            continue
        Rb, Tb = R[b.r0:b.r1, b.c0:b.c1], Rt[b.r0:b.r1, b.c0:b.c1]
        err = np.linalg.norm(Tb - Rb, 2)
        if b.kind == "rk":
            assert err <= 2 * tol * np.linalg.norm(Rb) + 1e-300, (b, err, np.linalg.norm(Rb))
        else:
            assert err <= 1e-12 * max(np.abs(Rb).max(), 1e-300)


def test_aca_matches_taylor_form_ranks():
    """The algebraic and the Taylor constructions, both recompressed to the same tolerance, need
    ranks of the same size and give the same matrix to that tolerance."""
    a = fh.HMatrix(0.5, 3.0, 1.0, 1024, 64, 0, 1e-10, lowrank="aca")
    b = fh.HMatrix(0.5, 3.0, 1.0, 1024, 64, 0, 1e-10)
    assert abs(a.info()["max_rank"] - b.info()["max_rank"]) <= 2
    Ra, Rb = a.dense(), b.dense()
    assert np.abs(Ra - Rb).max() <= 1e-9 * np.abs(Rb).max()


def test_aca_rejects_without_tolerance():
    with pytest.raises(fh.FhmgError):
        fh.HMatrix(0.5, 3.0, 1.0, 256, 64, 0, 0.0, lowrank="aca")
