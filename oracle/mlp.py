"""CPU oracle of the row-size predictor (test infrastructure only).

Not part of the paper: the library adds a small multilayer perceptron that
predicts log(1 + nnz(C_i)) of each output row from six row features, to size
hash tables and C's allocation without the exact symbolic pass. This file is
the plain float64 definition the GPU kernels are checked against:

  x  = (f - mean) * inv_std                      6 normalised features
  h1 = relu(W1 x + b1)                           W1: 64 x 6
  h2 = relu(W2 h1 + b2)                          W2: 64 x 64
  y  = w3 . h2 + b3
  loss = mean over the batch of (y - t)^2

and its gradient by the chain rule. Parameters are one flat vector in the
order W1 (row-major), b1, W2 (row-major), b2, w3, b3 (4673 values), the same
layout the library uses. Only tests import this module.
"""
from __future__ import annotations

import numpy as np

H = 64
F = 6
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, k = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[k:k + n].reshape(shape)
        k += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(p, x):
    """x: (n, 6) normalised features -> y (n,), plus the activations."""
    w = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ w["W1"].T + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w["w3"] + w["b3"][0]
    return y, (x, a1, h1, a2, h2)


def loss_and_grad(p, x, t):
    """Mean squared error and its gradient with respect to the flat parameters."""
    w = unpack(p)
    y, (x, a1, h1, a2, h2) = forward(p, x)
    n = x.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dh2 = np.outer(dy, w["w3"]) * (a2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ w["W2"]) * (a1 > 0)
    g["W1"] = dh1.T @ x
    g["b1"] = dh1.sum(axis=0)
    return loss, pack(g)


def normalise(feats, mean, inv_std):
    return (np.asarray(feats, dtype=np.float64) - mean) * inv_std
