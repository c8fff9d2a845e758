"""The tcgen05 walk (BF16 H-matrix products, FP32 accumulation in tensor memory, FP32 grid
functions) against the oracle, element by element, and the FHMG_MIXED_BF16 solves.

Error bound of one walk, derived from the arithmetic: the chunk entries and the x / y / z operands
are rounded to BF16 (8 significant bits, unit roundoff 2^-8), their products are exact in FP32, the
tensor core sums them into FP32 accumulators (each MMA step may lose about 2^-22 of the running
magnitude to alignment, and a row takes at most M/16 + 16 steps), and the diagonal of the diagonal
leaves (and of the level inverses) is applied in FP32.  So a product Y = R~ X deviates from the exact
one by at most
    2^-7 |D'| |X| + 2^-6 |U| |V|^T |X| + (M/16 + 16) 2^-22 (|R~| + |U| |V|^T) |X|,
D' the dense blocks without the diagonal (two roundings per term), U V^T the low-rank blocks (four:
V, x, z, U).  The line solve X = (R~ + sI)^-1 B deviates by at most |(R~ + sI)^-1| times the product
bound of its off-diagonal-block part at X plus |A_bd| times the error of the BF16 inverse product
(2^-7 |Dinv'| |Y| + ...), A_bd the diagonal leaf blocks of R~ + sI, Y = A_bd X (first order).  An exact
BF16 emulation of these steps in numpy reaches 0.6-0.8 of these bounds on the cases below.  Full
solves keep the FP64-accurate outer defect, so they reach the same 1e-7 bar as the FP32 form.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, hmatrix, l1  # noqa: E402
from paper_1706_07632_gb300 import inputs, warmstart  # noqa: E402

DEV = "cuda"
NCOLS = 128 * 152 + 1029  # enough 128-column tiles for every SM, and a ragged last tile


def f32(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device=DEV)


def time_matrix(alpha, gamma, M, rank, tol):
    """The time matrix both sides use (dense R, or the paper's rank-k Taylor form), with |D'| (dense
    blocks without the diagonal) and |U||V|^T of the low-rank blocks for the bounds."""
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    Rt = R
    lr = np.zeros_like(R)
    dense = np.tril(np.ones_like(R)) * R
    if rank > 0:
        Rt, blocks = hmatrix.approximate(t, alpha, R, 64, rank)
        dense = np.zeros_like(R)
        for b in blocks:
            if b.kind == "dense":
                dense[b.r0:b.r1, b.c0:b.c1] = Rt[b.r0:b.r1, b.c0:b.c1]
            elif b.kind == "rk":
                A, Bf = hmatrix.rk_factors(t, alpha, b, rank)
                lr[b.r0:b.r1, b.c0:b.c1] = np.abs(A) @ np.abs(Bf).T
    dense_off = np.abs(dense)
    np.fill_diagonal(dense_off, 0.0)
    return Rt, dense_off, lr


def product_bound(Rt, dense_off, lr, X):
    M = Rt.shape[0]
    steps = M / 16 + 16
    aX = np.abs(X)
    return 2.0 ** -7 * (dense_off @ aX) + 2.0 ** -6 * (lr @ aX) + steps * 2.0 ** -22 * ((np.abs(Rt) + lr) @ aX)


def solve_bound(Rt, dense_off, lr, X, s):
    M = Rt.shape[0]
    A = Rt + s * np.eye(M)
    Abd = np.zeros_like(A)
    inv_off = np.zeros_like(A)
    inv_abs = np.zeros_like(A)
    off_bd = dense_off.copy()
    for i in range(M // 64):
        sl = slice(64 * i, 64 * (i + 1))
        Abd[sl, sl] = A[sl, sl]
        Di = np.abs(np.linalg.inv(A[sl, sl]))
        inv_abs[sl, sl] = Di
        inv_off[sl, sl] = Di - np.diag(np.diag(Di))
        off_bd[sl, sl] = 0.0
    Y = np.abs(Abd @ X)
    inv_err = 2.0 ** -7 * (inv_off @ Y) + 20 * 2.0 ** -22 * (inv_abs @ Y)
    return np.abs(np.linalg.inv(A)) @ (product_bound(Rt, off_bd, lr, X) + np.abs(Abd) @ inv_err)


# (alpha, gamma, M, rank, tol): dense R, the paper's Taylor form
CASES = [(0.55, 2.0, 512, 0, 0.0), (0.4, 2.5, 256, 12, 0.0), (0.3, 1.7 / 0.3, 512, 10, 0.0)]


@pytest.mark.parametrize("case", CASES)
def test_umma_matvec_against_oracle(case):
    alpha, gamma, M, rank, tol = case
    Rt, dense_off, lr = time_matrix(alpha, gamma, M, rank, tol)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, rank, tol)
    P = fh.Problem(H, 1, 63, 1.0, fh.MIXED_BF16)
    X = inputs.random_field(11, (M, NCOLS)).astype(np.float32).astype(np.float64)
    Y = torch.empty((M, NCOLS), dtype=torch.float32, device=DEV)
    P.hmatvec_s(Y, f32(X))
    diff = np.abs(Y.cpu().numpy().astype(np.float64) - Rt @ X)
    bound = product_bound(Rt, dense_off, lr, X)
    assert np.all(diff <= bound), float((diff / bound).max())


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("level", [0, 5])
def test_umma_line_solve_against_oracle(case, level):
    alpha, gamma, M, rank, tol = case
    Rt, dense_off, lr = time_matrix(alpha, gamma, M, rank, tol)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, rank, tol)
    P = fh.Problem(H, 1, 63, 1.0, fh.MIXED_BF16)
    s = 2.0 * (2 ** (level + 1)) ** 2  # 2/h^2 on level `level` of the 63-point grid
    Bm = inputs.random_field(12, (M, NCOLS)).astype(np.float32).astype(np.float64)
    X = torch.empty((M, NCOLS), dtype=torch.float32, device=DEV)
    P.line_solve_s(level, X, f32(Bm))
    Xd = direct.solve_o2_mode(Rt, s, Bm)
    diff = np.abs(X.cpu().numpy().astype(np.float64) - Xd)
    bound = solve_bound(Rt, dense_off, lr, Xd, s) + 2.0 ** -22 * np.abs(Xd)
    assert np.all(diff <= bound), float((diff / bound).max())


def test_umma_used_only_on_wide_panels_and_narrow_ones_match_fp32():
    """Below 128 x SMs columns the BF16 problem falls back to the FP32 products: the same result as
    an FHMG_MIXED_FP32 problem, to FP32 rounding."""
    alpha, gamma, M = 0.5, 2.0, 256
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    Pb = fh.Problem(H, 1, 63, 1.0, fh.MIXED_BF16)
    Pf = fh.Problem(H, 1, 63, 1.0, fh.MIXED_FP32)
    X = f32(inputs.random_field(13, (M, 2000)))
    Yb = torch.empty_like(X)
    Yf = torch.empty_like(X)
    Pb.hmatvec_s(Yb, X)
    Pf.hmatvec_s(Yf, X)
    assert float((Yb - Yf).abs().max() / Yf.abs().max()) < 1e-5


@pytest.mark.parametrize("dim,N,M,alpha,gamma", [(2, 255, 256, 0.5, 2.0), (2, 511, 1024, 0.4, 2.5)])
def test_bf16_solve_manufactured_against_oracle(dim, N, M, alpha, gamma):
    """Mixed BF16 solve of the manufactured source to relres 1e-8: within 1e-7 of the per-mode
    oracle (the 511^2 x 1024 case is the 2D workload)."""
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    h = 1.0 / (N + 1)
    a, s = inputs.manufactured(t[1:], N, dim, alpha)
    w = direct.solve_o2_mode(R, dim * direct.laplacian_eigs_1d(N, h)[0], a)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, dim, N, 1.0, fh.MIXED_BF16)
    P.set_coarse_direct(31)
    dv = torch.as_tensor
    f = dv(a, device=DEV)[:, None, None] * dv(s, device=DEV)[None]
    u = torch.zeros_like(f)
    k, rr = P.solve(u, f, None, 1, 1, 1e-8, 60)
    ref = dv(w, device=DEV)[:, None, None] * dv(s, device=DEV)[None]
    err = float((u - ref).abs().max() / ref.abs().max())
    assert rr <= 1e-8 and err < 1e-7, (k, rr, err)


def test_bf16_solve_warmstart_workload_against_oracle():
    """2D N=1023^2, M=512, alpha=0.55, GRF source, relres 1e-8 of max|F|: the BF16 form against the
    per-mode oracle at 2048 sampled grid points (1e-7)."""
    alpha, gamma, M, N, seed = 0.55, 2.0, 512, 1023, 41
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    t, _ = H.mesh()
    f = warmstart.source_field(2, seed, t[1:], N)
    P = fh.Problem(H, 2, N, 1.0, fh.MIXED_BF16)
    P.set_coarse_direct(31)
    P.set_rtol_reference(1)
    u = torch.zeros_like(f)
    k, rr = P.solve(u, f, None, 1, 1, 1e-8, 60)
    R = l1.l1_matrix(l1.graded_mesh(1.0, M, gamma), alpha)
    _, _, c = inputs.grf_2d(seed, t[1:], N)
    lam = direct.laplacian_eigs_1d(N, 1.0 / (N + 1))
    x = inputs.grid(N)
    rng = np.random.default_rng(3)
    iy, ix = rng.integers(0, N, 2048), rng.integers(0, N, 2048)
    ref = np.zeros((M, 2048))
    for p in range(c.shape[0]):
        for q in range(c.shape[1]):
            if c[p, q] != 0.0:
                wv = direct.solve_o2_mode(R, lam[p] + lam[q], np.full(M, c[p, q]))
                ref += np.outer(wv, np.sin((p + 1) * math.pi * x[iy]) * np.sin((q + 1) * math.pi * x[ix]))
    got = u[:, torch.as_tensor(iy, device=DEV), torch.as_tensor(ix, device=DEV)].cpu().numpy()
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    assert rr <= 1e-8 and err < 1e-7, (k, rr, err)


def test_umma_timeout_is_reported_and_cleared():
    """The tcgen05 walk's bounded waits: a withheld chunk makes them give up; the call that reads the
    error word reports FHMG_ETIMEOUT, tensor memory was released (later launches allocate it
    again), and the next walk gives the clean result."""
    H = fh.HMatrix(0.5, 2.0, 1.0, 256, 64, 0, 1e-10)
    P = fh.Problem(H, 1, 63, 1.0, fh.MIXED_BF16)
    X = f32(inputs.random_field(14, (256, NCOLS)))
    Y0 = torch.empty_like(X)
    P.hmatvec_s(Y0, X)
    P.inject_timeout(512)
    Y1 = torch.empty_like(X)
    P.hmatvec_s(Y1, X)
    f = torch.zeros((256, 63), dtype=torch.float64, device=DEV)
    with pytest.raises(fh.FhmgError) as e:
        P.residual_norm(f, f)
    assert e.value.status == fh.FHMG_ETIMEOUT
    Y2 = torch.empty_like(X)
    P.hmatvec_s(Y2, X)
    assert float((Y2 - Y0).abs().max()) == 0.0
