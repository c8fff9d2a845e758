"""Learned warm start: data generation by the solver, training and prediction (orchestration only).

Every numerical step runs in the library: the solves that produce the training solutions
(fhmg_solve), their projection onto the leading sine modes (fhmg_ws_dataset), training
(fhmg_wsnet_train: FP32 forward/backward/Adam kernels) and prediction (fhmg_ws_predict: feature,
network (BF16 tensor cores), synthesis kernels).  This module chooses sizes and seeds, orders
the training rows at random (a host-side permutation) and runs the learning-rate schedule.

The warm start predicts, for a source constant in time and a finite sine series, the per-mode
response lam_k w_k(t) with (R + lam_k I) w_k = 1 -- a function of lam, alpha and the time mesh
only, so a network trained on a small grid with the same M and gamma serves larger grids.
"""
from __future__ import annotations

import numpy as np

from . import FP64, MIXED_FP32, HMatrix, Problem, WSNet, inputs, ws_dataset


def _source(dim, seed, t, N, ell):
    if dim == 2:
        a, s, _ = inputs.grf_2d(seed, t, N, ell)
    else:
        a, s, _ = inputs.sine_series_1d(seed, t, N)
    return a, s


def generate(dim, N, M, gamma, alphas, seeds, K=24, ell=0.1, prec=MIXED_FP32, rtol=1e-10, device="cuda"):
    """Training pairs from library solves of random smooth sources (one per (alpha, seed))."""
    import torch
    Xs, Ys = [], []
    for alpha, seed in zip(alphas, seeds):
        H = HMatrix(alpha, gamma, 1.0, M, 64, 0, 1e-10)
        P = Problem(H, dim, N, 1.0, prec)
        t, _ = H.mesh()
        a, s = _source(dim, seed, t[1:], N, ell)
        f = torch.as_tensor(a, device=device).reshape((-1,) + (1,) * dim) * torch.as_tensor(s, device=device)[None]
        u = torch.zeros_like(f)
        P.solve(u, f, None, 1, 1, rtol, 60, allow_notconv=True)
        # modes whose source coefficient is tiny carry no usable target (their amplitude is at the
        # solver's noise level): keep |c_k| >= 1e-3 max |c|
        X, Y = ws_dataset(P, u, f, alpha, K, rel_thr=1e-3)
        Xs.append(X.cpu().numpy())
        Ys.append(Y.cpu().numpy())
        del P, H, f, u
    X = np.concatenate(Xs)
    Y = np.concatenate(Ys)
    perm = np.random.default_rng(12345).permutation(len(Y))
    return (torch.as_tensor(np.ascontiguousarray(X[perm]), device=device),
            torch.as_tensor(np.ascontiguousarray(Y[perm]), device=device))


def train(net: WSNet, X, Y, steps=4000, batch=4096, lr=2e-3, seed=0):
    """Adam with a step-down schedule (lr, lr/4, lr/16 over the thirds of the run); returns the
    last mini-batch loss of each phase."""
    losses = []
    for k, scale in enumerate((1.0, 0.25, 0.0625)):
        losses.append(net.train(X, Y, batch=min(batch, X.shape[0]), steps=steps // 3, lr=lr * scale, seed=seed + k))
    return losses


def source_field(dim, seed, t, N, ell=0.1, device="cuda"):
    """The random smooth source of a seed on the problem's time levels, as a device tensor."""
    import torch
    a, s = _source(dim, seed, t, N, ell)
    return torch.as_tensor(a, device=device).reshape((-1,) + (1,) * dim) * torch.as_tensor(s, device=device)[None]
