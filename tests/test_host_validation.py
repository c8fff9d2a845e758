"""Argument validation of the host-only entry points (no GPU): every invalid argument is refused
with FHMG_EINVAL and a message before any work, nothing is created, and the degenerate but valid
sizes (one leaf, M = leaf) are accepted."""
import ctypes

import numpy as np
import pytest

import paper_1706_07632_gb300 as fh
from oracle import l1


def einval(fn, *args):
    with pytest.raises(fh.FhmgError) as e:
        fn(*args)
    assert e.value.status == fh.FHMG_EINVAL
    assert len(str(e.value)) > len("FHMG_EINVAL: ")


@pytest.mark.parametrize("alpha,gamma,T,M,leaf,rank,tol", [
    (0.0, 2.0, 1.0, 256, 64, 0, 1e-10),     # alpha outside (0, 1)
    (1.0, 2.0, 1.0, 256, 64, 0, 1e-10),
    (0.5, 0.9, 1.0, 256, 64, 0, 1e-10),     # gamma < 1
    (0.5, 2.0, 0.0, 256, 64, 0, 1e-10),     # T <= 0
    (0.5, 2.0, 1.0, 384, 64, 0, 1e-10),     # M not leaf * 2^p
    (0.5, 2.0, 1.0, 256, 48, 0, 1e-10),     # leaf not 16, 32, 64
    (0.5, 2.0, 1.0, 256, 64, 65, 0.0),      # rank > 64
    (0.5, 2.0, 1.0, 256, 64, 0, -1e-10),    # tol < 0
])
def test_build_hmatrix_rejects(alpha, gamma, T, M, leaf, rank, tol):
    einval(fh.HMatrix, alpha, gamma, T, M, leaf, rank, tol)


@pytest.mark.parametrize("tol,M,leaf", [(0.0, 256, 64), (1e-10, 384, 64), (1e-10, 256, 40)])
def test_build_hmatrix_aca_rejects(tol, M, leaf):
    einval(lambda: fh.HMatrix(0.5, 2.0, 1.0, M, leaf, 0, tol, lowrank="aca"))


def test_null_output_pointers_are_refused():
    L = fh.lib()
    assert L.fhmg_build_hmatrix(0.5, 2.0, 1.0, 64, 64, 0, 0.0, None) == fh.FHMG_EINVAL
    H = fh.HMatrix(0.5, 2.0, 1.0, 128, 64, 0, 0.0)
    assert L.fhmg_hmatrix_split_digits(H._h, None, None, None, None) == fh.FHMG_EINVAL
    assert L.fhmg_hmatrix_dense(H._h, None) == fh.FHMG_EINVAL
    # a tile buffer smaller than the tiles is refused, not overrun
    n = ctypes.c_longlong(0)
    assert L.fhmg_hmatrix_split_digits(H._h, None, ctypes.byref(n), None, None) == fh.FHMG_OK
    assert n.value > 1
    buf = np.zeros((n.value - 1, 8192), dtype=np.uint16)
    small = ctypes.c_longlong(n.value - 1)
    assert L.fhmg_hmatrix_split_digits(H._h, buf.ctypes.data, ctypes.byref(small), None, None) == fh.FHMG_EINVAL
    assert not buf.any()


@pytest.mark.parametrize("dim,N,nu1,nu2", [(3, 63, 1, 1), (2, 64, 1, 1), (1, 1, 1, 1), (2, 63, 0, 0)])
def test_sama_rejects(dim, N, nu1, nu2):
    H = fh.HMatrix(0.5, 2.0, 1.0, 64, 64, 0, 0.0)
    einval(H.sama_two_grid, dim, N, 1.0, nu1, nu2)


@pytest.mark.parametrize("M,leaf", [(16, 64), (32, 32), (64, 64)])
def test_single_leaf_sizes_are_valid(M, leaf):
    """M <= leaf: one diagonal leaf (no low-rank block), R~ = R exactly."""
    H = fh.HMatrix(0.6, 1.5, 1.0, M, leaf, 0, 1e-10)
    info = H.info()
    assert info["n_lowrank"] == 0 and info["n_dense"] == 1
    t = l1.graded_mesh(1.0, M, 1.5)
    Ro = l1.l1_matrix(t, 0.6)
    R = H.dense()
    nz = Ro != 0
    assert np.all(R[~nz] == 0)
    assert np.max(np.abs(R[nz] - Ro[nz]) / np.abs(Ro[nz])) < 1e-12
