"""Reference implementation of the warm-start network (oracle; test infrastructure only).

Plain numpy, FP64: the same architecture and parameter layout as the library's network (6 input
features -> `hidden` x `layers` SiLU layers -> 1 linear output; parameters layer by layer, W_l
row-major (n_{l+1} x n_l) then b_l), the mean-squared loss, and its gradient by explicit
backpropagation.  The gradient is pinned by central finite differences
(tests/test_oracle_nn.py), and the GPU kernels' gradients are checked against it.

Features of a mode with eigenvalue lam, order alpha and time t (s = lam t^alpha):
log10(lam)/5, alpha, log10(t)/5, s/(1+s), log1p(s)/10, t^alpha.
"""
from __future__ import annotations

import numpy as np

NFEAT = 6


def features(lam, alpha, t):
    lam, t = np.broadcast_arrays(np.asarray(lam, dtype=np.float64), np.asarray(t, dtype=np.float64))
    ta = t ** alpha
    s = lam * ta
    return np.stack([np.log10(lam) / 5.0, np.full(lam.shape, alpha), np.log10(t) / 5.0,
                     s / (1.0 + s), np.log1p(s) / 10.0, ta], axis=-1)


def widths(hidden, layers):
    return [NFEAT] + [hidden] * layers + [1]


def unpack(params, w):
    out, off = [], 0
    for l in range(len(w) - 1):
        W = params[off:off + w[l + 1] * w[l]].reshape(w[l + 1], w[l])
        off += w[l + 1] * w[l]
        b = params[off:off + w[l + 1]]
        off += w[l + 1]
        out.append((W, b))
    assert off == len(params)
    return out


def _silu(z):
    return z / (1.0 + np.exp(-z))


def forward(params, w, X):
    a = np.asarray(X, dtype=np.float64)
    layers = unpack(np.asarray(params, dtype=np.float64), w)
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        a = _silu(z) if l < len(layers) - 1 else z
    return a[:, 0]


def loss_grad(params, w, X, Y):
    """mean (y - Y)^2 and its gradient with respect to the flat parameter vector."""
    params = np.asarray(params, dtype=np.float64)
    layers = unpack(params, w)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = X.shape[0]
    acts, zs = [X], []
    a = X
    for l, (W, b) in enumerate(layers):
        z = a @ W.T + b
        zs.append(z)
        a = _silu(z) if l < len(layers) - 1 else z
        acts.append(a)
    y = a[:, 0]
    loss = np.mean((y - Y) ** 2)
    grads = []
    d = (2.0 * (y - Y) / n)[:, None]            # dL/d(output pre-activation), last layer linear
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        if l < len(layers) - 1:
            z = zs[l]
            sg = 1.0 / (1.0 + np.exp(-z))
            d = d * sg * (1.0 + z * (1.0 - sg))  # SiLU'
        grads.append((d.T @ acts[l], d.sum(axis=0)))
        d = d @ W
    grads.reverse()
    return loss, np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
