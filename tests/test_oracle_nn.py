"""Pins for oracle.nn: the backpropagated gradient against central finite differences, and the
feature map against direct evaluation."""
import math

import numpy as np

from oracle import nn


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = nn.widths(7, 2)
    nparam = sum(w[l + 1] * w[l] + w[l + 1] for l in range(len(w) - 1))
    p = rng.standard_normal(nparam) * 0.5
    X = rng.standard_normal((13, nn.NFEAT))
    Y = rng.standard_normal(13)
    loss, g = nn.loss_grad(p, w, X, Y)
    assert abs(loss - np.mean((nn.forward(p, w, X) - Y) ** 2)) < 1e-14
    eps = 1e-6
    fd = np.empty_like(p)
    for i in range(nparam):
        e = np.zeros_like(p)
        e[i] = eps
        fd[i] = (nn.loss_grad(p + e, w, X, Y)[0] - nn.loss_grad(p - e, w, X, Y)[0]) / (2 * eps)
    assert np.max(np.abs(fd - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_features_direct():
    f = nn.features(np.array([9.8696, 1000.0]), 0.5, np.array([0.25, 1.0]))
    assert f.shape == (2, 6)
    s = 9.8696 * 0.5
    assert math.isclose(f[0, 0], math.log10(9.8696) / 5)
    assert math.isclose(f[0, 3], s / (1 + s)) and math.isclose(f[0, 4], math.log1p(s) / 10)
    assert math.isclose(f[1, 2], 0.0, abs_tol=1e-15) and math.isclose(f[1, 5], 1.0)
