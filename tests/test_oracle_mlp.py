"""Pins for oracle/mlp.py: exact gradients by central finite differences; BF16 rounding."""
import numpy as np

from oracle import mlp


def _params(seed=0, scale=0.05):
    rng = np.random.default_rng(seed)
    w = rng.uniform(-scale, scale, mlp.NPARAM)
    W1 = w[mlp.OFF_W1:mlp.OFF_B1].reshape(mlp.HID, mlp.IN_PAD)
    W1[:, mlp.IN:] = 0.0
    return w


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    w = _params(1, 0.2)
    X = rng.standard_normal((3, mlp.IN))
    T = rng.standard_normal((3, mlp.OUT))
    _, g = mlp.grads(w, X, T)
    idx = np.concatenate([rng.integers(mlp.OFF_W1, mlp.OFF_B1, 12), rng.integers(mlp.OFF_B1, mlp.OFF_W2, 4),
                          rng.integers(mlp.OFF_W2, mlp.OFF_B2, 8), rng.integers(mlp.OFF_B2, mlp.OFF_W3, 4),
                          rng.integers(mlp.OFF_W3, mlp.OFF_B3, 8), rng.integers(mlp.OFF_B3, mlp.NPARAM, 4)])
    for i in idx:
        if mlp.OFF_W1 <= i < mlp.OFF_B1 and (i - mlp.OFF_W1) % mlp.IN_PAD >= mlp.IN:
            continue
        h = 1e-5
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss(wp, X, T) - mlp.loss(wm, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_gelu_derivative_and_bf16_rounding():
    z = np.linspace(-4, 4, 101)
    h = 1e-6
    assert np.allclose((mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), mlp.gelu_grad(z), atol=1e-8)
    # bfloat16 keeps 8 significand bits: 1 + 2^-8 rounds to even (1.0), 1 + 3*2^-8 to 1 + 2^-6
    assert mlp.to_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert mlp.to_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    x = np.random.default_rng(2).standard_normal(1000)
    assert np.max(np.abs(mlp.to_bf16(x) - x) / np.abs(x)) <= 2 ** -8
