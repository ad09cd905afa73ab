"""Pins of the oracle's FP64 cost-model twin (CPU only): central finite
differences for the gradient, the closed form of Adam's first step, a zero
learning rate, fitting a handful of rows, and hand-bucketed segment lengths
for the length histogram."""
import numpy as np

import synth
from oracle import mlp


def _data(F, B, seed):
    X = synth.normal_f32(B * F, seed=seed).numpy().reshape(B, F).astype(np.float64)
    t = synth.normal_f32(B, seed=seed + 1).numpy().astype(np.float64)
    return X, t


def test_gradient_matches_finite_differences():
    F, H, B = 6, 8, 10
    p = synth.mlp_init(F, H, seed=1).double().numpy()
    p[H * F:H * F + H] = 0.05        # nonzero biases
    X, t = _data(F, B, 2)
    _, g = mlp.backward(p, X, t, F, H)
    h = 1e-6
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, X, t, F, H) - mlp.loss(p - e, X, t, F, H)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_adam_first_step_closed_form():
    # after one step m_hat = g and v_hat = g^2, so the update is lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p0 = np.array([1.0, 1.0, 1.0, 1.0])
    p1, m, v = mlp.adam(p0, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_zero_learning_rate_is_a_no_op():
    F, H = 4, 8
    p = synth.mlp_init(F, H, seed=3).double().numpy()
    X, t = _data(F, 8, 4)
    _, g = mlp.backward(p, X, t, F, H)
    p1, _, _ = mlp.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr=0.0)
    assert np.array_equal(p1, p)


def test_fits_eight_rows():
    F, H = 5, 16
    p = synth.mlp_init(F, H, seed=5).double().numpy()
    X, t = _data(F, 8, 6)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = mlp.loss(p, X, t, F, H)
    for step in range(1, 3001):
        _, g = mlp.backward(p, X, t, F, H)
        p, m, v = mlp.adam(p, g, m, v, step, lr=3e-3)
    assert mlp.loss(p, X, t, F, H) < 1e-3 * l0


def test_length_histogram_hand_buckets():
    # floor(log2 L): 0 -> bucket 0 (empty), 1 -> 0 (bucket 0), 7 -> 2 (bucket 0), 8 -> 3 (bucket 1),
    # 63 -> 5 (bucket 1), 64 -> 6 (bucket 2), 511 -> 8 (bucket 2), 2^20 -> 20 (bucket 6),
    # 2^23 -> 23 (bucket 7), 2^30 -> 30 (bucket 7)
    L = [0, 1, 7, 8, 63, 64, 1 << 20, 1 << 23, 1 << 30, 511]
    h = mlp.length_histogram(L)
    assert h == [0.3, 0.2, 0.2, 0.0, 0.0, 0.0, 0.1, 0.2]
    assert mlp.length_histogram([]) == [0.0] * 8
    assert abs(sum(mlp.length_histogram(range(1, 5000))) - 1.0) < 1e-12
