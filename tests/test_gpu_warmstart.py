"""Warm-start network: gradients of the GPU kernels against the CPU oracle, BF16 inference (against
FP32 and against a BF16 emulation), the training pairs against per-mode oracle solutions, and the
cycles the trained network saves."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1706_07632_gb300 as fh  # noqa: E402
from oracle import direct, l1, nn  # noqa: E402
from paper_1706_07632_gb300 import inputs, warmstart  # noqa: E402

DEV = "cuda"


def test_gradient_matches_oracle():
    net = fh.WSNet(48, 3, seed=7)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((1000, 6)).astype(np.float32)
    Y = rng.standard_normal(1000).astype(np.float32)
    loss, g = net.loss_grad(torch.as_tensor(X, device=DEV), torch.as_tensor(Y, device=DEV))
    p = net.get_params().astype(np.float64)
    loss_o, g_o = nn.loss_grad(p, nn.widths(48, 3), X, Y)
    assert abs(loss - loss_o) <= 1e-5 * loss_o
    assert np.max(np.abs(g - g_o)) <= 1e-4 * np.max(np.abs(g_o))
    # forward values too
    y = torch.empty(1000, dtype=torch.float32, device=DEV)
    net.forward(torch.as_tensor(X, device=DEV), y)
    yo = nn.forward(p, nn.widths(48, 3), X)
    assert np.max(np.abs(y.cpu().numpy() - yo)) <= 1e-5 * np.max(np.abs(yo))


def test_bf16_inference_close_to_fp32():
    net = fh.WSNet(320, 3, seed=1)
    assert 150_000 <= net.num_params() <= 250_000
    rng = np.random.default_rng(4)
    X = torch.as_tensor(rng.uniform(-1, 1, (3000, 6)).astype(np.float32), device=DEV)
    y32 = torch.empty(3000, dtype=torch.float32, device=DEV)
    y16 = torch.empty_like(y32)
    net.forward(X, y32)
    net.forward(X, y16, bf16=True)
    assert float((y32 - y16).abs().max()) <= 3e-2 * float(y32.abs().max())


def _bf16(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("hidden,n", [(320, 3001), (320, 100), (64, 777)])
def test_bf16_inference_matches_bf16_emulation(hidden, n):
    """BF16 inference (hidden layers on the tiled tensor-core kernel with bias and SiLU fused,
    ragged row counts) against a layer-by-layer emulation: inputs, weights and every hidden
    activation rounded to BF16, products summed in FP64.  The kernel sums in FP32, so an activation
    may round to the neighbouring BF16 value; 5e-3 of max|y| bounds that and fails for any
    misplaced fragment or row."""
    net = fh.WSNet(hidden, 3, seed=5)
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, (n, 6)).astype(np.float32)
    y16 = torch.empty(n, dtype=torch.float32, device=DEV)
    net.forward(torch.as_tensor(X, device=DEV), y16, bf16=True)
    layers = nn.unpack(net.get_params().astype(np.float64), nn.widths(hidden, 3))
    a = _bf16(X)
    for l, (W, b) in enumerate(layers):
        z = a @ _bf16(W).T + b
        if l < len(layers) - 1:
            a = _bf16((z / (1.0 + np.exp(-z))).astype(np.float32))
        else:
            a = z
    y = a[:, 0]
    assert float(np.max(np.abs(y16.cpu().numpy() - y))) <= 5e-3 * float(np.max(np.abs(y)))


def test_training_pairs_match_mode_solutions():
    """For a sine-series source the multigrid solution carries each mode as c_k w_k(t) with
    (R + lam_k I) w_k = 1: the projected targets lam_k w_k must match the oracle's solves."""
    alpha, gamma, M, N, K = 0.55, 2.0, 64, 31, 8
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 0.0)
    P = fh.Problem(H, 2, N)
    t, _ = H.mesh()
    f = warmstart.source_field(2, 5, t[1:], N, 0.25)
    u = torch.zeros_like(f)
    P.solve(u, f, None, 1, 1, 1e-11, 40, allow_notconv=True)
    X, Y = fh.ws_dataset(P, u, f, alpha, K, rel_thr=1e-3)
    X = X.cpu().numpy()
    Y = Y.cpu().numpy()
    to = l1.graded_mesh(1.0, M, gamma)
    R = l1.l1_matrix(to, alpha)
    lam_all = []
    h = 1.0 / (N + 1)
    for p in range(1, K + 1):
        for q in range(1, K + 1):
            lam_all.append(4 / h ** 2 * (math.sin(p * math.pi * h / 2) ** 2 + math.sin(q * math.pi * h / 2) ** 2))
    lam_all = np.array(lam_all)
    rows = len(Y) // M
    assert rows >= 4
    for r in range(rows):
        lam = 10 ** (5 * X[r * M, 0])
        k = int(np.argmin(np.abs(lam_all - lam)))
        w = direct.solve_o2_mode(R, lam_all[k], np.ones(M))
        assert np.max(np.abs(Y[r * M:(r + 1) * M] - lam_all[k] * w)) <= 2e-3, r
    # the features of the first row agree with the oracle's feature map
    fo = nn.features(lam_all[int(np.argmin(np.abs(lam_all - 10 ** (5 * X[0, 0]))))], alpha, to[1:])
    assert np.max(np.abs(X[:M] - fo)) <= 1e-5


def test_trained_warm_start_saves_cycles():
    dim, N, M, gamma = 2, 63, 128, 2.0
    alphas = [0.3, 0.4, 0.5, 0.6, 0.7, 0.8]
    X, Y = warmstart.generate(dim, N, M, gamma, alphas, seeds=list(range(10, 16)), K=24, prec=fh.FP64)
    net = fh.WSNet(320, 3, seed=0)
    losses = warmstart.train(net, X, Y, steps=3000, batch=4096, lr=2e-3)
    assert losses[-1] < 1e-4
    alpha = 0.55
    H = fh.HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
    P = fh.Problem(H, dim, N, 1.0, fh.FP64)
    P.set_rtol_reference(1)
    t, _ = H.mesh()
    f = warmstart.source_field(dim, 99, t[1:], N)
    u0 = torch.zeros_like(f)
    k0, _ = P.solve(u0, f, None, 1, 1, 1e-8, 40)
    uw = net.predict(P, f, alpha, K=24, bf16=True)
    kw, _ = P.solve(uw, f, None, 1, 1, 1e-8, 40)
    assert kw < k0, (kw, k0)
    # multigrid decides on the warm start: both iterates meet the same absolute defect target
    assert float((uw - u0).abs().max() / u0.abs().max()) < 1e-6
