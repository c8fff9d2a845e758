"""The tcgen05 walk (BF16 H-matrix products, FP32 accumulation in tensor memory, FP32 grid
functions) against the oracle, element by element, and the FHMG_MIXED_BF16 solves.

Error bound of one walk, derived from the arithmetic: the chunk entries and the x / y / z operands
are rounded to BF16 (relative error <= 2^-9 each), their products are exact in FP32 and summed in
FP32; the diagonal of the diagonal leaves (and of the level inverses) is applied in FP32.  So a
product Y = R~ X deviates from the exact one by at most (2 * 2^-9 + 2^-18) |R~'| |X| plus FP32
rounding (a few 2^-24 |R~| |X| per leaf), R~' = R~ without its diagonal; the line solve
X = (R~ + sI)^-1 B by at most |(R~ + sI)^-1| times that product bound evaluated at X (first order;
the tests allow a factor 2).  Full solves keep the FP64-accurate outer defect, so they reach the
same 1e-7 bar as the FP32 form.
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
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    if rank > 0:
        return t, hmatrix.approximate(t, alpha, R, 64, rank)[0]
    return t, R


# (alpha, gamma, M, rank, tol): dense R, the paper's Taylor form
CASES = [(0.55, 2.0, 512, 0, 0.0), (0.4, 2.5, 256, 12, 0.0), (0.3, 1.7 / 0.3, 512, 10, 0.0)]


@pytest.mark.parametrize("case", CASES)
def test_umma_matvec_against_oracle(case):
    alpha, gamma, M, rank, tol = case
    t, Rt = time_matrix(*case)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, rank, tol)
    P = fh.Problem(H, 1, 63, 1.0, fh.MIXED_BF16)
    X = inputs.random_field(11, (M, NCOLS)).astype(np.float32).astype(np.float64)
    Y = torch.empty((M, NCOLS), dtype=torch.float32, device=DEV)
    P.hmatvec_s(Y, f32(X))
    exact = Rt @ X
    off = np.abs(Rt - np.diag(np.diag(Rt)))
    bound = (2 * 2.0 ** -9 + 2.0 ** -18) * (off @ np.abs(X)) + 2.0 ** -18 * (np.abs(Rt) @ np.abs(X))
    diff = np.abs(Y.cpu().numpy().astype(np.float64) - exact)
    assert np.all(diff <= bound), float((diff / bound).max())


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("level", [0, 5])
def test_umma_line_solve_against_oracle(case, level):
    alpha, gamma, M, rank, tol = case
    t, Rt = time_matrix(*case)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, rank, tol)
    P = fh.Problem(H, 1, 63, 1.0, fh.MIXED_BF16)
    s = 2.0 * (2 ** (level + 1)) ** 2  # 2/h^2 on level `level` of the 63-point grid
    Bm = inputs.random_field(12, (M, NCOLS)).astype(np.float32).astype(np.float64)
    X = torch.empty((M, NCOLS), dtype=torch.float32, device=DEV)
    P.line_solve_s(level, X, f32(Bm))
    A = Rt + s * np.eye(M)
    Xd = direct.solve_o2_mode(Rt, s, Bm)
    off = np.abs(Rt - np.diag(np.diag(Rt)))
    Ainv = np.abs(np.linalg.inv(A))
    # the product bound at Xd, propagated through |A^-1|, plus the inverse's own BF16 products
    prod = (2 * 2.0 ** -9 + 2.0 ** -18) * (off @ np.abs(Xd)) + 2.0 ** -18 * (np.abs(A) @ np.abs(Xd))
    inv_off = np.abs(np.linalg.inv(A) - np.diag(np.diag(np.linalg.inv(A))))
    bound = 2.0 * (Ainv @ prod + (2 * 2.0 ** -9) * (inv_off @ np.abs(A @ Xd)))
    diff = np.abs(X.cpu().numpy().astype(np.float64) - Xd)
    assert np.all(diff <= bound + 1e-30), float((diff / (bound + 1e-30)).max())


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
