"""The outer defect by digit splitting on the tcgen05 tensor cores (defect arithmetic 2) against
the oracle, element by element.

Error bound (derived from the arithmetic): R~ and u are split per time row / per grid point into
7 balanced base-2^7 digits after rounding to 49 bits relative to 2^E_m > max_k |R~_mk| and
2^F_c > max_k |u_kc|.  Per term k the rounding of both factors costs <= 2^{E_m + F_c - 49} and the
dropped digit groups (a + b >= 7) <= 2^{E_m + F_c - 48.4}; the group sums are exact integers in the
FP32 accumulators except the last group, whose accumulation loses at most 2^{E_m + F_c - 48.2}
per output; the double-float combination of the groups adds a few 2^-47 of |R~||u|; the stencil and
the subtractions run in FP64 (a few 2^-53 of |A_h||u| + |F| -- fine grids need it: at N = 4095 the
stencil cancels 2^24-fold).  With a factor 2 of margin:
    |r - r_oracle| <= (m + 2) 2^{E_m + F_c - 46} + 2^-45 |R~||u| + 2^-50 (|A_h||u| + |F|).
The time matrix is the paper's rank-k Taylor form (or dense R), which the oracle builds itself.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, hmatrix, l1  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402

DEV = "cuda"


def abs_stencil(u, h):
    """|A_h| |u| (the stencil with absolute values), time-major grid functions."""
    a = np.abs(u)
    dim = u.ndim - 1
    s = 2.0 * dim * a
    for ax in range(1, u.ndim):
        lo = [slice(None)] * u.ndim
        hi = [slice(None)] * u.ndim
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        s[tuple(lo)] += a[tuple(hi)]
        s[tuple(hi)] += a[tuple(lo)]
    return s / h ** 2


def split_bound(Rt, u, F, h):
    M = Rt.shape[0]
    E = np.array([math.frexp(float(np.abs(Rt[m]).max()))[1] for m in range(M)], dtype=float)
    U = u.reshape(M, -1)
    Fc = np.array([math.frexp(float(x))[1] for x in np.abs(U).max(axis=0)], dtype=float)
    trunc = (np.arange(M) + 2.0)[:, None] * np.exp2(E[:, None] + Fc[None, :] - 46.0)
    prod = np.abs(Rt) @ np.abs(U)
    sten = abs_stencil(u, h).reshape(M, -1) + np.abs(F).reshape(M, -1)
    return (trunc + 2.0 ** -45 * prod + 2.0 ** -50 * sten).reshape(u.shape)


def time_matrix(alpha, gamma, M, leaf, rank):
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    return (hmatrix.approximate(t, alpha, R, leaf, rank)[0] if rank else R), t


# (dim, N, M, alpha, gamma, rank): ragged last tiles (65,025 = 1016 x 64 + 1 points; 4095 points),
# one to four output blocks of 128 time rows, dense R and the Taylor form
CASES = [(2, 255, 512, 0.55, 2.0, 12), (2, 127, 256, 0.3, 1.7 / 0.3, 10), (1, 4095, 128, 0.8, 1.5, 0),
         (2, 63, 128, 0.5, 3.0, 0)]


@pytest.mark.parametrize("dim,N,M,alpha,gamma,rank", CASES)
@pytest.mark.parametrize("prec", [fh.MIXED_FP32, fh.MIXED_BF16])
def test_split_defect_against_oracle(dim, N, M, alpha, gamma, rank, prec):
    Rt, t = time_matrix(alpha, gamma, M, 64, rank)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, rank, 0.0)
    P = fh.Problem(H, dim, N, 1.0, prec)
    h = 1.0 / (N + 1)
    shape = (M,) + (N,) * dim
    # a smooth-in-time iterate with the solution's t^alpha layer, plus noise; F of unit size
    prof = (t[1:] ** alpha)[(slice(None),) + (None,) * dim]
    u = prof * (1.0 + 0.1 * inputs.random_field(31, shape))
    F = inputs.random_field(32, shape)
    r = torch.empty(shape, dtype=torch.float64, device=DEV)
    P.residual(torch.as_tensor(u, device=DEV), torch.as_tensor(F, device=DEV), None, r)
    ref = direct.residual(Rt, F, u, h)
    diff = np.abs(r.cpu().numpy() - ref)
    bound = split_bound(Rt, u, F, h)
    assert np.all(diff <= bound), float((diff / bound).max())


@pytest.mark.parametrize("prec", [fh.MIXED_FP32, fh.MIXED_BF16])
def test_split_solve_fine_1d_reaches_target(prec):
    """1D N = 4095 (the stencil cancels 2^24-fold), M = 512: the mixed solve with the split defect
    reaches relres 1e-8 and the per-mode oracle's solution to 1e-7 (a double-float stencil, 2^-48, would
    leave the residual floor above 1e-8 here)."""
    alpha, gamma, M, N = 0.8, 1.5, 512, 4095
    t = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(t, alpha)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 1, N, 1.0, prec)
    assert P.split_flops() is not None
    a, sx = inputs.manufactured(t[1:], N, 1, alpha)
    w = direct.solve_o2_mode(R, direct.laplacian_eigs_1d(N, 1.0 / (N + 1))[0], a)
    f = torch.as_tensor(np.outer(a, sx), device=DEV)
    u = torch.zeros_like(f)
    k, rr = P.solve(u, f, None, 1, 1, 1e-8, 60)
    ref = np.outer(w, sx)
    err = float(np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max())
    assert rr <= 1e-8 and err < 1e-7, (k, rr, err)


def test_split_matches_double_float_defect():
    """The same problem with defect arithmetic 1 (double-float walk): both FP64-accurate, so they
    agree within the sum of their bounds (here 1e-12 of the defect's max-norm)."""
    alpha, gamma, M, N = 0.55, 2.0, 512, 255
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 2, N, 1.0, fh.MIXED_BF16)
    t, _ = H.mesh()
    shape = (M, N, N)
    u = torch.as_tensor((t[1:] ** alpha)[:, None, None] * inputs.random_field(33, shape), device=DEV)
    F = torch.as_tensor(inputs.random_field(34, shape), device=DEV)
    r2 = torch.empty_like(u)
    r1 = torch.empty_like(u)
    P.residual(u, F, None, r2)
    P.set_defect_arith(1)
    P.residual(u, F, None, r1)
    P.set_defect_arith(2)
    scale = float(r1.abs().max())
    assert float((r2 - r1).abs().max()) <= 1e-12 * scale


def test_split_extreme_values_and_nan():
    """Grid points whose values span 2^-300 .. 2^300 across time levels and points, zero columns,
    and a NaN: finite outputs within the bound, and a NaN max-norm once u holds a NaN."""
    alpha, gamma, M, N = 0.5, 2.0, 256, 63
    Rt, t = time_matrix(alpha, gamma, M, 64, 0)
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 0.0)
    P = fh.Problem(H, 2, N, 1.0, fh.MIXED_FP32)
    h = 1.0 / (N + 1)
    shape = (M, N, N)
    rng = np.random.default_rng(35)
    expo = rng.integers(-300, 300, size=(1, N, N)).astype(float)
    u = rng.standard_normal(shape) * np.exp2(expo) * np.exp2(rng.integers(-20, 0, size=(M, 1, 1)))
    u[:, 5, :] = 0.0
    F = rng.standard_normal(shape)
    r = torch.empty(shape, dtype=torch.float64, device=DEV)
    P.residual(torch.as_tensor(u, device=DEV), torch.as_tensor(F, device=DEV), None, r)
    ref = direct.residual(Rt, F, u, h)
    diff = np.abs(r.cpu().numpy() - ref)
    bound = split_bound(Rt, u, F, h)
    assert np.all(diff <= bound), float((diff / bound).max())
    u[7, 3, 4] = float("nan")
    assert math.isnan(P.residual_norm(torch.as_tensor(u, device=DEV), torch.as_tensor(F, device=DEV)))


def test_split_timeout_is_reported_and_cleared():
    """A withheld digit tile makes the bounded waits give up: FHMG_ETIMEOUT once, tensor memory
    released, then the clean defect again."""
    H = fh.HMatrix(0.5, 2.0, 1.0, 256, 64, 0, 1e-10)
    P = fh.Problem(H, 2, 127, 1.0, fh.MIXED_BF16)
    shape = (256, 127, 127)
    u = torch.as_tensor(inputs.random_field(36, shape), device=DEV)
    F = torch.as_tensor(inputs.random_field(37, shape), device=DEV)
    n0 = P.residual_norm(u, F)
    P.inject_timeout(512)
    with pytest.raises(fh.FhmgError) as e:
        P.residual_norm(u, F)
    assert e.value.status == fh.FHMG_ETIMEOUT
    assert P.residual_norm(u, F) == n0


def test_split_arith_rejected_where_unavailable():
    H = fh.HMatrix(0.5, 2.0, 1.0, 1024, 64, 0, 1e-10)
    P = fh.Problem(H, 1, 63, 1.0, fh.MIXED_FP32)
    with pytest.raises(fh.FhmgError):
        P.set_defect_arith(2)
    P64 = fh.Problem(fh.HMatrix(0.5, 2.0, 1.0, 256, 64, 0, 1e-10), 1, 63, 1.0, fh.FP64)
    with pytest.raises(fh.FhmgError):
        P64.set_defect_arith(2)
