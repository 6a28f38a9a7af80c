"""CPU reference of the learned form's per-element MLP (forward, loss, gradients).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network (the learned form of the method's hot path, not a paper equation): 586
inputs -> 128 -> 128 -> 192, GELU(z) = z/2 (1 + erf(z/sqrt 2)) after both hidden
layers, loss = mean over rows and outputs of (Y - T)^2. Parameters are one flat
vector laid out as W1 [128][592] (input padded with 6 zero columns), b1, W2
[128][128], b2, W3 [192][128], b3.

`grads(..., bf16=False)` is the exact FP64 gradient (pinned by central finite
differences in tests/test_oracle_mlp.py). `bf16=True` rounds to bfloat16 (round
to nearest even) at the points where the GPU kernels store BF16: the packed
input, both hidden activations, the output gradient and both pre-activation
gradients, and the weights used in the products -- everything else stays FP64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

IN, IN_PAD, HID, OUT = 586, 592, 128, 192
OFF_W1 = 0
OFF_B1 = OFF_W1 + HID * IN_PAD
OFF_W2 = OFF_B1 + HID
OFF_B2 = OFF_W2 + HID * HID
OFF_W3 = OFF_B2 + HID
OFF_B3 = OFF_W3 + OUT * HID
NPARAM = OFF_B3 + OUT


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) and return as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(w: np.ndarray):
    w = np.asarray(w, dtype=np.float64)
    W1 = w[OFF_W1:OFF_B1].reshape(HID, IN_PAD)
    W2 = w[OFF_W2:OFF_B2].reshape(HID, HID)
    W3 = w[OFF_W3:OFF_B3].reshape(OUT, HID)
    return W1, w[OFF_B1:OFF_W2], W2, w[OFF_B2:OFF_W3], W3, w[OFF_B3:NPARAM]


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(w, X, bf16=False):
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(w)
    Xp = np.zeros((X.shape[0], IN_PAD))
    Xp[:, :IN] = X
    Xp = r(Xp)
    Z1 = Xp @ r(W1).T + b1
    H1 = r(gelu(Z1))
    Z2 = H1 @ r(W2).T + b2
    H2 = r(gelu(Z2))
    Y = H2 @ r(W3).T + b3
    return Y, (Xp, Z1, H1, Z2, H2)


def loss(w, X, T, bf16=False):
    Y, _ = forward(w, X, bf16)
    return float(np.mean((Y - T) ** 2))


def grads(w, X, T, bf16=False):
    """Loss and its gradient with respect to the flat parameter vector."""
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(w)
    Y, (Xp, Z1, H1, Z2, H2) = forward(w, X, bf16)
    n = X.shape[0]
    dY = r(2.0 * (Y - T) / (n * OUT))
    g = np.zeros(NPARAM)
    g[OFF_W3:OFF_B3] = (dY.T @ H2).ravel()
    g[OFF_B3:NPARAM] = dY.sum(axis=0)
    dZ2 = r((dY @ r(W3)) * gelu_grad(Z2))
    g[OFF_W2:OFF_B2] = (dZ2.T @ H1).ravel()
    g[OFF_B2:OFF_W3] = dZ2.sum(axis=0)
    dZ1 = r((dZ2 @ r(W2)) * gelu_grad(Z1))
    g[OFF_W1:OFF_B1] = (dZ1.T @ Xp).ravel()
    g[OFF_B1:OFF_W2] = dZ1.sum(axis=0)
    return float(np.mean((Y - T) ** 2)), g
