"""Pins of the FP64 surrogate MLP reference: its gradient against central finite
differences, its forward pass against an independent evaluation, and the bfloat16
rounding helper against torch."""
import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(rng)
    x = rng.standard_normal((5, 36))
    t = rng.standard_normal((5, 128))
    _, g = mlp.loss_and_grad(theta, x, t)
    idx = rng.choice(theta.size, 300, replace=False)
    # include parameters of every tensor
    bounds = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    idx = np.concatenate([idx, bounds[:-1], bounds[1:] - 1])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, x, t)[0] - mlp.loss_and_grad(tm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_forward_by_loops():
    rng = np.random.default_rng(1)
    theta = mlp.init_params(rng)
    x = rng.standard_normal((2, 36))
    W1, b1, W2, b2, W3, b3, W4, b4 = mlp.unpack(theta)
    y, _ = mlp.forward(theta, x)
    for s in range(2):
        h = x[s]
        for W, b, act in ((W1, b1, True), (W2, b2, True), (W3, b3, True), (W4, b4, False)):
            out = np.array([sum(W[o, i] * h[i] for i in range(W.shape[1])) + b[o] for o in range(W.shape[0])])
            h = np.maximum(out, 0.0) if act else out
        assert np.allclose(h, y[s], rtol=1e-12, atol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    a = np.concatenate([rng.standard_normal(1000) * 10 ** rng.uniform(-5, 5, 1000), [0.0, -0.0, 1.0, 3.0e38]])
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)
    assert np.array_equal(mlp.to_bf16(a), ref)
