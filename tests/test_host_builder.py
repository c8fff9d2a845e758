"""Host-side H-matrix builder of the library (no GPU) against the oracle: mesh, initial-data
weights, dense L1 entries, the paper's Taylor factors, and the recompressed form."""
import math

import numpy as np
import pytest

import paper_1706_07632_gb300 as fh
from oracle import direct, hmatrix, l1


@pytest.mark.parametrize("alpha,gamma,M", [(0.5, 2.0, 64), (0.3, 1.7 / 0.3, 256), (0.8, 1.0, 128)])
def test_mesh_weights_and_dense_R(alpha, gamma, M):
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 0.0)      # dense mode
    t, dmm = H.mesh()
    to = l1.graded_mesh(1.0, M, gamma)
    assert np.max(np.abs(t - to)) <= 4e-16 * np.abs(to).max()
    assert np.allclose(dmm, l1.initial_coeff(to, alpha), rtol=1e-13, atol=0)
    R = H.dense()
    Ro = l1.l1_matrix(to, alpha)
    nz = Ro != 0
    assert np.all(R[~nz] == 0)
    assert np.max(np.abs(R[nz] - Ro[nz]) / np.abs(Ro[nz])) < 1e-12


@pytest.mark.parametrize("alpha,gamma,k", [(0.5, 2.0, 8), (0.3, 1.7 / 0.3, 12), (0.8, 1.5, 20)])
def test_taylor_mode_matches_oracle_taylor(alpha, gamma, k):
    """rank = k: the paper's Section 3 factors, no recompression."""
    M, leaf = 512, 32
    H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, k, 0.0)
    to = l1.graded_mesh(1.0, M, gamma)
    Ro = l1.l1_matrix(to, alpha)
    Rt_o, blocks = hmatrix.approximate(to, alpha, Ro, leaf, k)
    info = H.info()
    assert info["n_lowrank"] == sum(b.kind == "rk" for b in blocks)
    assert info["n_dense"] == sum(b.kind == "dense" for b in blocks)
    Rt = H.dense()
    scale = np.abs(Ro).max(axis=1, keepdims=True)
    assert np.max(np.abs(Rt - Rt_o) / scale) < 1e-12


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
def test_recompressed_within_tolerance(alpha):
    M, leaf, tol = 1024, 64, 1e-10
    gamma = (2 - alpha) / alpha
    H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, 0, tol)
    to = l1.graded_mesh(1.0, M, gamma)
    Ro = l1.l1_matrix(to, alpha)
    Rt = H.dense()
    blocks = hmatrix.block_tree(to, leaf)
    for b in blocks:
        if b.kind != "rk":
            continue
        blk = Ro[b.r0:b.r1, b.c0:b.c1]
        err = np.linalg.norm(Rt[b.r0:b.r1, b.c0:b.c1] - blk, 2)
        assert err <= 20 * tol * np.linalg.norm(blk, 2)
    assert 2 <= H.info()["max_rank"] <= 16
    # the perturbed discrete solution stays within 1e-8 of the dense one (single mode, N=4095)
    N = 4095
    h = 1.0 / (N + 1)
    lam = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    Ft = math.gamma(1 + alpha) + math.pi ** 2 * to[1:] ** alpha
    w = direct.solve_o2_mode(Ro, lam, Ft)
    wt = direct.solve_o2_mode(Rt, lam, Ft)
    assert np.abs(wt - w).max() <= 1e-8 * np.abs(w).max()
