"""GPU parity of the double-float defect products (fhmg_hmatvec_df; the mixed path's FP64-accurate
outer defect) against the FP64 oracle and the FP64 (DFMA) walk, element by element.

Tolerance: entries and x are split into float pairs with |a - hi - lo| <= 2^-48 |a|; a product adds
hi*hi exactly and the cross terms with FP32 rounding, and sums keep a float pair, so a dot
product is exact to a few 2^-48 (3.6e-15) of sum |a_k x_k|.  On these inputs sum |R x| is at most
a few tens of |R x|: bar 3e-13 relative max-norm (the FP64 walk agrees with numpy to ~1e-15)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, hmatrix, l1  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402

DEV = "cuda"

# dense R (no far blocks), dense R with near-field blocks beyond the ring, the paper's Taylor form,
# the recompressed H-matrix, leaf 32
MODES = [
    (0.5, 2.0, 256, 64, 0, 0.0),
    (0.8, 1.5, 1024, 64, 0, 0.0),
    (0.3, 1.7 / 0.3, 512, 64, 12, 0.0),
    (0.5, 3.0, 2048, 64, 0, 1e-10),
    (0.4, 2.5, 1024, 32, 0, 1e-10),
]


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def host(x):
    torch.cuda.synchronize()
    return x.cpu().numpy()


_cache = {}


def setup(mode):
    if mode not in _cache:
        alpha, gamma, M, leaf, rank, tol = mode
        H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, rank, tol)
        P = fh.Problem(H, 1, 7, prec=fh.MIXED_FP32)
        R = None
        if tol == 0.0:
            t = l1.graded_mesh(1.0, M, gamma)
            R = l1.l1_matrix(t, alpha)
            if rank > 0:
                R = hmatrix.approximate(t, alpha, R, leaf, rank)[0]
        _cache[mode] = (H, P, R)
    return _cache[mode]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("tile", [0, 4, 8, 16])
@pytest.mark.parametrize("ncols", [37, 1029])
def test_df_product(mode, tile, ncols):
    H, P, R = setup(mode)
    M = mode[2]
    X = dev(inputs.random_field(41, (M, ncols)))
    Y = torch.empty_like(X)
    Y64 = torch.empty_like(X)
    P.hmatvec_df(Y, X, tile)
    P.hmatvec(Y64, X)
    y, y64 = host(Y), host(Y64)
    assert rel(y, y64) < 3e-13
    if R is not None:
        assert rel(y, R @ host(X)) < 3e-13


def test_df_needs_a_mixed_problem():
    H = fh.HMatrix(0.5, 2.0, 1.0, 64, 64, 0, 0.0)
    P = fh.Problem(H, 1, 7)
    X = torch.zeros((64, 3), dtype=torch.float64, device=DEV)
    with pytest.raises(fh.FhmgError):
        P.hmatvec_df(X.clone(), X, 0)


def test_mixed_solve_same_with_fp64_and_double_float_defects():
    """1D N=4095, M=4096: the mixed solve takes the same cycles with either arithmetic for the outer
    defect and the coarse mode solves, and both solutions match the per-mode oracle to 1e-7."""
    alpha, gamma, M, N = 0.5, 3.0, 4096, 4095
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    h = 1.0 / (N + 1)
    lam = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    a, s = inputs.manufactured(t[1:], N, 1, alpha)
    w = direct.solve_o2_mode(R, lam, a)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    f = dev(a)[:, None] * dev(s)[None, :]
    ref = torch.as_tensor(w, device=DEV)[:, None] * dev(s)[None, :]
    out = []
    for arith in (0, 1):
        P = fh.Problem(H, 1, N, prec=fh.MIXED_FP32)
        P.set_coarse_direct(255)
        P.set_defect_arith(arith)
        u = torch.zeros((M, N), dtype=torch.float64, device=DEV)
        k, rr = P.solve(u, f, None, 1, 1, 1e-8, 30)
        err = float((u - ref).abs().max() / ref.abs().max())
        assert rr <= 1e-8 and err < 1e-7, (arith, k, rr, err)
        out.append((k, rr, u))
    # arithmetic 1 also runs the exactly solved level's mode solves in double-float: the coarse
    # corrections then differ at the 1e-13 level and the FP32-product inner cycles carry that into
    # the iterates, so the two solutions agree to the solve's tolerance, not bit for bit
    assert out[0][0] == out[1][0]
    assert abs(out[0][1] - out[1][1]) <= 0.5 * out[0][1]
    assert float((out[0][2] - out[1][2]).abs().max() / ref.abs().max()) < 1e-9


@pytest.mark.parametrize("dim,N,nc", [(1, 127, 31), (2, 31, 7)])
def test_vcycle_with_double_float_mode_solves(dim, N, nc):
    """A mixed-precision problem's FP64 V-cycle (fhmg_vcycle) solves the exact coarse level's modes in
    double-float arithmetic: one cycle against the oracle's cycle with the same coarse correction."""
    from oracle import wrmg
    alpha, gamma, M = 0.5, 2.0, 256
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 0.0)
    P = fh.Problem(H, dim, N, prec=fh.MIXED_FP32)
    P.set_coarse_direct(nc)
    shape = (M, N) if dim == 1 else (M, N, N)
    u0 = inputs.random_field(42, shape)
    F = inputs.random_field(43, shape) * 10
    u = dev(u0)
    P.vcycle(u, dev(F), None, 1, 1)
    ref = wrmg.cycle(R, F, u0, 1.0 / (N + 1), 1, 1, n_direct=nc)
    assert rel(host(u), ref) < 1e-11
