"""FP64 reference of the surrogate MLP -- TEST INFRASTRUCTURE ONLY.

Linear(n_in, H) - GELU - Linear(H, H) - GELU - Linear(H, n_out), loss = mean
squared error over batch x outputs.  Plain numpy in float64.  With
``bf16=True`` every tensor that the GPU rounds to bfloat16 before a matrix
product (inputs, weights, hidden activations, backward deltas) is rounded the
same way (round to nearest even), so the GPU's gradients can be compared with
this code on the same rounded tensors.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def to_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return (b.astype(np.uint32).view(np.float32)).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(p, x, bf16=False):
    W1, b1, W2, b2, W3, b3 = p
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    X = r(x)
    Z1 = X @ r(W1).T + b1
    H1 = r(gelu(Z1))
    Z2 = H1 @ r(W2).T + b2
    H2 = r(gelu(Z2))
    Y = H2 @ r(W3).T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss_and_grads(p, x, t, bf16=False):
    W1, b1, W2, b2, W3, b3 = p
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    Y, (X, Z1, H1, Z2, H2) = forward(p, x, bf16)
    n = Y.size
    loss = float(np.sum((Y - t) ** 2) / n)
    dY = r(2.0 * (Y - t) / n)
    gW3 = dY.T @ H2
    gb3 = dY.sum(0)
    dZ2 = r((dY @ r(W3)) * gelu_grad(Z2))
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(0)
    dZ1 = r((dZ2 @ r(W2)) * gelu_grad(Z1))
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(0)
    return loss, [gW1, gb1, gW2, gb2, gW3, gb3]
