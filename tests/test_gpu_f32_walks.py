"""GPU parity of the mixed path's FP32-product walks (SIMT kernel for every column tile, tensor-core
kernel for tiles 16 and 32 with leaf 64) against the FP64 oracle, element by element.

Tolerance: the products use FP32 matrix entries and x tiles (relative rounding 6e-8) and FP32
accumulation over at most a few hundred terms per leaf row, so a product R~ X is exact to a few
1e-7 of max|R~ X|; a line solve propagates that through the triangular recurrence.  Bars: 2e-6
(products) and 2e-5 (solves), relative max-norm; the tensor-core split in three TF32 products is held
to the same bars and to 1e-5 against the SIMT kernel."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, hmatrix, l1  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402

DEV = "cuda"

# (alpha, gamma, M, leaf, rank, tol): recompressed H, the paper's Taylor form (larger U/V slabs),
# dense lower triangle with near-field blocks beyond the ring (tensor cores fall back to SIMT)
MODES = [
    (0.5, 3.0, 1024, 64, 0, 1e-10),
    (0.3, 1.7 / 0.3, 512, 64, 12, 0.0),
    (0.8, 1.5, 1024, 64, 0, 0.0),
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
        t = l1.graded_mesh(1.0, M, gamma)
        R = l1.l1_matrix(t, alpha)
        Rt = hmatrix.approximate(t, alpha, R, leaf, rank)[0] if rank > 0 else R
        H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, rank, tol)
        P = fh.Problem(H, 1, 63, prec=fh.MIXED_FP32)
        _cache[mode] = (Rt, H, P)
    return _cache[mode]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("tile", [0, 1, 2, 8, 16, 32])
@pytest.mark.parametrize("ncols", [37, 1029])
def test_f32_line_solve(mode, tile, ncols):
    Rt, H, P = setup(mode)
    M = mode[2]
    B = inputs.random_field(31, (M, ncols))
    X = torch.empty((M, ncols), dtype=torch.float64, device=DEV)
    for level in (0, 5):
        h = 1.0 / (2 ** (level + 1))
        P.line_solve_f32(level, X, dev(B), tile)
        assert rel(host(X), direct.solve_o2_mode(Rt, 2.0 / h ** 2, B)) < 2e-5


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("tile", [0, 1, 4, 16, 32])
def test_f32_hmatvec(mode, tile):
    Rt, H, P = setup(mode)
    M, ncols = mode[2], 517
    X = inputs.random_field(32, (M, ncols))
    Y = torch.empty((M, ncols), dtype=torch.float64, device=DEV)
    P.hmatvec_f32(Y, dev(X), tile)
    assert rel(host(Y), Rt @ X) < 2e-6


@pytest.mark.parametrize("tile", [16, 32])
def test_tensor_cores_match_simt(tile):
    Rt, H, P = setup(MODES[0])
    M, ncols = MODES[0][2], 2000
    B = dev(inputs.random_field(33, (M, ncols)))
    X1 = torch.empty_like(B)
    X2 = torch.empty_like(B)
    P.set_tensor_cores(True)
    P.line_solve_f32(3, X1, B, tile)
    P.hmatvec_f32(X2, B, tile)
    P.set_tensor_cores(False)
    Y1 = torch.empty_like(B)
    Y2 = torch.empty_like(B)
    P.line_solve_f32(3, Y1, B, tile)
    P.hmatvec_f32(Y2, B, tile)
    P.set_tensor_cores(True)
    assert rel(host(X1), host(Y1)) < 1e-5
    assert rel(host(X2), host(Y2)) < 1e-5


def test_f32_entry_points_need_a_mixed_problem():
    H = fh.HMatrix(0.5, 2.0, 1.0, 64, 64, 0, 0.0)
    P = fh.Problem(H, 1, 7)
    X = torch.zeros((64, 3), dtype=torch.float64, device=DEV)
    with pytest.raises(fh.FhmgError):
        P.line_solve_f32(0, X, X.clone(), 0)


@pytest.mark.parametrize("tc", [True, False])
def test_full_size_mixed_solve_with_and_without_tensor_cores(tc):
    """1D N=4095, M=4096, alpha=.5: the mixed solve reaches 1e-8 with either product kernel and
    matches the per-mode oracle to 1e-7."""
    import math
    alpha, gamma, M, N = 0.5, 3.0, 4096, 4095
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    h = 1.0 / (N + 1)
    lam = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    a, s = inputs.manufactured(t[1:], N, 1, alpha)
    w = direct.solve_o2_mode(R, lam, a)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 1, N, prec=fh.MIXED_FP32)
    P.set_tensor_cores(tc)
    P.set_coarse_direct(255)
    f = dev(a)[:, None] * dev(s)[None, :]
    u = torch.zeros((M, N), dtype=torch.float64, device=DEV)
    k, rr = P.solve(u, f, None, 1, 1, 1e-8, 30)
    assert rr <= 1e-8
    ref = torch.as_tensor(w, device=DEV)[:, None] * dev(s)[None, :]
    err = float((u - ref).abs().max() / ref.abs().max())
    assert err < 1e-7, (tc, err, k, rr)
