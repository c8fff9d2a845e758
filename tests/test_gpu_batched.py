"""Batched solves (many instances, one launch per stage, graph-captured cycles) and the
autotuner, against single-instance solves and the oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, l1  # noqa: E402
from paper_1706_07632_gb300 import inputs  # noqa: E402

DEV = "cuda"


def _instances(seed, n, leaves=(64,)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        alpha = float(rng.uniform(0.2, 0.9))
        gamma = float(rng.uniform(1.0, 3.0))
        M = int(rng.choice([64, 128, 256]))
        N = int(rng.choice([63, 127, 255]))
        leaf = leaves[i % len(leaves)]
        out.append((alpha, gamma, M, N, leaf))
    return out


def _setup(inst, prec, seed0=0):
    Hs, Ps, us, fs, fnp = [], [], [], [], []
    for i, (alpha, gamma, M, N, leaf) in enumerate(inst):
        H = fh.HMatrix(alpha, gamma, 1.0, M, leaf, 0, 1e-10)
        P = fh.Problem(H, 1, N, 1.0, prec)
        t, _ = H.mesh()
        a, s, c = inputs.sine_series_1d(seed0 + i, t[1:], N)
        f = np.outer(a, s)
        Hs.append(H)
        Ps.append(P)
        fnp.append(f)
        fs.append(torch.as_tensor(f, device=DEV))
        us.append(torch.zeros((M, N), dtype=torch.float64, device=DEV))
    return Hs, Ps, us, fs, fnp


@pytest.mark.parametrize("leaves", [(64,), (32, 64)])
def test_batched_fp64_matches_single_solves(leaves):
    inst = _instances(1, 9, leaves)
    Hs, Ps, us, fs, fnp = _setup(inst, fh.FP64)
    k_b, rr_b = fh.solve_batched(Ps, us, fs, 1, 1, 1e-8, 60)
    for i, (alpha, gamma, M, N, leaf) in enumerate(inst):
        u1 = torch.zeros_like(us[i])
        k1, rr1 = Ps[i].solve(u1, fs[i], None, 1, 1, 1e-8, 60)
        assert k_b[i] == k1
        assert float((us[i] - u1).abs().max() / u1.abs().max()) < 1e-11
        t = l1.graded_mesh(1.0, M, gamma)
        ud = direct.solve_o1(l1.l1_matrix(t, alpha), fnp[i], 1.0 / (N + 1))
        assert float(np.abs(us[i].cpu().numpy() - ud).max() / np.abs(ud).max()) < 1e-6
        assert rr_b[i] <= 1e-8


def test_batched_mixed_reaches_tolerance():
    inst = _instances(2, 12, (64,))
    Hs, Ps, us, fs, fnp = _setup(inst, fh.MIXED_FP32, seed0=100)
    k_b, rr_b = fh.solve_batched(Ps, us, fs, 1, 1, 1e-8, 60)
    for i, (alpha, gamma, M, N, leaf) in enumerate(inst):
        assert rr_b[i] <= 1e-8
        t = l1.graded_mesh(1.0, M, gamma)
        R = l1.l1_matrix(t, alpha)
        uh = us[i].cpu().numpy()
        r = direct.residual(R, fnp[i], uh, 1.0 / (N + 1))
        assert np.abs(r).max() <= 2e-8 * np.abs(fnp[i]).max()


def test_autotune_keeps_results_and_picks_a_leaf():
    alpha, gamma, M, N = 0.5, 2.0, 256, 255
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, 1, N)
    t, _ = H.mesh()
    a, s = inputs.manufactured(t[1:], N, 1, alpha)
    f = torch.as_tensor(np.outer(a, s), device=DEV)
    u0 = torch.zeros_like(f)
    P.solve(u0, f, None, 1, 1, 1e-9, 40)
    P.autotune()
    u1 = torch.zeros_like(f)
    P.solve(u1, f, None, 1, 1, 1e-9, 40)
    assert float((u1 - u0).abs().max() / u0.abs().max()) < 1e-11
    leaf, ms = fh.autotune_leaf(alpha, gamma, 1.0, M, 1e-10, 1, N)
    assert leaf in (16, 32, 64) and ms > 0
