"""Oracle: FP64 twin of the schedule cost model (test infrastructure).

The paper has no learned component; the cost model is an addition of this
library.  Its definition, restated here independently of the CUDA kernels:

  h1 = relu(W1 x + b1)        W1: H x F
  h2 = relu(W2 h1 + b2)       W2: H x H
  y  = w3 . h2 + b3           w3: H, b3 scalar       (predicts log time)
  L  = (1/B) sum_i (y_i - t_i)^2

relu'(z) is 1 for z > 0 and 0 otherwise.  Parameters are one flat vector
[W1 (row-major), b1, W2 (row-major), b2, w3, b3].  The optimiser is Adam
(Kingma and Ba 2015, Algorithm 1) with bias correction.  One group of input
features is the segment-length histogram of a batched call
(length_histogram below).
"""
from __future__ import annotations

import numpy as np


def n_params(F, H):
    return H * F + H + H * H + H + H + 1


def unpack(p, F, H):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, X, F, H):
    """Predictions y (B,) and the activations needed by backward."""
    W1, b1, W2, b2, w3, b3 = unpack(p, F, H)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    return y, (X, z1, h1, z2, h2)


def loss(p, X, t, F, H):
    y, _ = forward(p, X, F, H)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def backward(p, X, t, F, H):
    """(loss, gradient of the loss w.r.t. the flat parameter vector)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, F, H)
    y, (X, z1, h1, z2, h2) = forward(p, X, F, H)
    B = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B
    dw3 = h2.T @ dy
    db3 = dy.sum()
    dz2 = np.outer(dy, w3) * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    dW1 = dz1.T @ X
    db1 = dz1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return float(np.mean((y - t) ** 2)), g


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; ``step`` counts from 1.  Returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def length_histogram(lengths):
    """The cost model's segment-length feature: for buckets b = 0..7, the
    fraction of segments whose length L has floor(log2 L) in [3b, 3b + 3)
    (the last bucket also takes every longer segment); empty segments count
    in bucket 0.  Written with integer bit lengths: floor(log2 L) is
    L.bit_length() - 1 for L >= 1."""
    counts = [0] * 8
    L = [int(v) for v in lengths]
    for v in L:
        b = 0 if v <= 0 else min((v.bit_length() - 1) // 3, 7)
        counts[b] += 1
    return [c / len(L) for c in counts] if L else [0.0] * 8
