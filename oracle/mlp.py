"""FP64 reference of the hydrograph surrogate MLP (test infrastructure only).

y = W4 r(W3 r(W2 r(W1 x + b1) + b2) + b3) + b4 with r = max(., 0), parameters packed as
W1 (256 x 36), b1, W2 (256 x 256), b2, W3, b3, W4 (128 x 256), b4; loss = mean of
(y - t)^2 over all batch x 128 outputs.  Plain numpy in float64: the forward pass as
written and its gradient by the chain rule, layer by layer; the same two passes with
every operand rounded to bfloat16 where a BF16 network stores it (the mixed-precision
form the GPU computes, so that its outputs can be compared element by element); and
one Adam step (Kingma and Ba, "Adam: a method for stochastic optimization", ICLR 2015,
Algorithm 1) with an L2 weight-decay term on the weight matrices.  Only tests load it.
The surrogate is not part of the paper; these definitions are the textbook ones.
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


def weight_mask():
    """1 for the entries of the weight matrices, 0 for the biases (packed layout)."""
    return pack([np.ones(sh) if len(sh) == 2 else np.zeros(sh) for sh in SHAPES])


def adam_step(theta, m, v, grad, t, lr, weight_decay=0.0, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in float64 (Kingma and Ba 2015, Algorithm 1), t = 1, 2, ... the
    step's index.  The L2 term weight_decay * theta is added to the gradient of the weight
    matrices only (not the biases) before the moments are updated:
        g' = g + wd theta (weights),  m = b1 m + (1 - b1) g',  v = b2 v + (1 - b2) g'^2,
        theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
    Returns (theta, m, v) as new arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64) + weight_decay * weight_mask() * theta
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def forward_bf16(theta, x):
    """The forward pass of a BF16 network with float accumulation: inputs and weights
    rounded to bfloat16, each hidden layer's pre-activation formed exactly (float64 here),
    the bias added, the ReLU applied and the result rounded to bfloat16 (the operand the
    next layer reads); the output layer's result is not rounded.  Returns y and the
    stored operands (x_b, a1, a2, a3) and the rounded weights (W1..W4 as bfloat16)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    Wb = [to_bf16(W) for W in (W1, W2, W3, W4)]
    xb = to_bf16(x)
    a1 = to_bf16(np.maximum(xb @ Wb[0].T + b1, 0.0))
    a2 = to_bf16(np.maximum(a1 @ Wb[1].T + b2, 0.0))
    a3 = to_bf16(np.maximum(a2 @ Wb[2].T + b3, 0.0))
    y = a3 @ Wb[3].T + b4
    return y, (xb, a1, a2, a3), Wb


def loss_and_grad_bf16(theta, x, t):
    """Loss and gradient of the BF16 network of forward_bf16: the output gradient
    dY = 2 (y - t) / n and each back-propagated dZ = (dZ_next W) r' are rounded to bfloat16
    (the operands of the next products), the ReLU derivative taken where the stored
    activation is positive; weight gradients dW = dZ^T A and bias gradients sum_m dZ are
    formed exactly from those operands.  Also returns, per packed parameter, the sum of
    the magnitudes of the terms of its gradient (sum |dZ| |A|, sum |dZ|): the scale an
    elementwise tolerance is stated against."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta)
    y, (xb, a1, a2, a3), Wb = forward_bf16(theta, x)
    t = np.asarray(t, dtype=np.float64)
    n = y.size
    loss = float(np.sum((y - t) ** 2) / n)
    dy = to_bf16(2.0 * (y - t) / n)
    dz3 = to_bf16((dy @ Wb[3]) * (a3 > 0))
    dz2 = to_bf16((dz3 @ Wb[2]) * (a2 > 0))
    dz1 = to_bf16((dz2 @ Wb[1]) * (a1 > 0))
    grads, scales = [], []
    for dz, a in ((dz1, xb), (dz2, a1), (dz3, a2), (dy, a3)):
        grads += [dz.T @ a, dz.sum(axis=0)]
        scales += [np.abs(dz).T @ np.abs(a), np.abs(dz).sum(axis=0)]
    return loss, pack(grads), pack(scales)
