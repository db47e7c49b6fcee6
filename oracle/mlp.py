"""FP64 reference of the hydrograph surrogate MLP (test infrastructure only).

y = W4 r(W3 r(W2 r(W1 x + b1) + b2) + b3) + b4 with r = max(., 0), parameters packed as
W1 (256 x 36), b1, W2 (256 x 256), b2, W3, b3, W4 (128 x 256), b4; loss = mean of
(y - t)^2 over all batch x 128 outputs.  Plain numpy in float64: the forward pass as
written and its gradient by the chain rule, layer by layer.  Only tests load it.
"""
from __future__ import annotations

import numpy as np

SHAPES = [(256, 36), (256,), (256, 256), (256,), (256, 256), (256,), (128, 256), (128,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64).reshape(-1)
    assert theta.size == N_PARAMS
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in parts])


def forward(theta, x):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    z3 = a2 @ W3.T + b3
    a3 = np.maximum(z3, 0.0)
    y = a3 @ W4.T + b4
    return y, (x, z1, a1, z2, a2, z3, a3)


def loss_and_grad(theta, x, t):
    """Mean-squared error and its gradient with respect to the packed parameters."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    y, (x, z1, a1, z2, a2, z3, a3) = forward(theta, x)
    t = np.asarray(t, dtype=np.float64)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    dy = 2.0 * (y - t) / n
    gW4 = dy.T @ a3
    gb4 = dy.sum(axis=0)
    dz3 = (dy @ W4) * (z3 > 0)
    gW3 = dz3.T @ a2
    gb3 = dz3.sum(axis=0)
    dz2 = (dz3 @ W3) * (z2 > 0)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(axis=0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4])


def init_params(rng, scale=1.0):
    """He-style initialisation (weights ~ N(0, 2 / fan_in) * scale, biases 0)."""
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            parts.append(rng.standard_normal(s) * np.sqrt(2.0 / s[1]) * scale)
        else:
            parts.append(np.zeros(s))
    return pack(parts)


def to_bf16(a):
    """Round float64/float32 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
