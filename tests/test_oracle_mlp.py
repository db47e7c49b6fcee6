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


# ---------------------------------------------------------------- Adam (Kingma and Ba 2015)
#
# Pins that follow from the algorithm rather than restate it: the bias corrections make the
# first step, and every step of a constant gradient, move each parameter by exactly
# lr g / (|g| + eps); a worked two-step case; the decay acts on the weight matrices only.

LR = 1e-3


def _bias_slice(k):
    bounds = np.cumsum([0] + [int(np.prod(s)) for s in mlp.SHAPES])
    return slice(int(bounds[k]), int(bounds[k + 1]))


def _adam_pins(adam_step):
    """Each pin returns True when it holds; the list is what a mutant must break."""
    rng = np.random.default_rng(11)
    theta = mlp.init_params(rng)
    z = np.zeros_like(theta)
    res = {}
    # first step: m_hat = g, v_hat = g^2, so d theta = -lr g / (|g| + eps), elementwise
    g = rng.standard_normal(theta.size) * 10.0 ** rng.uniform(-6, 1, theta.size)
    th1, m1, v1 = adam_step(theta, z, z, g, 1, LR)
    res["first_step"] = np.allclose(th1 - theta, -LR * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
    # a gradient comparable to eps: d theta = -lr / 2 exactly when g = eps
    th1, _, _ = adam_step(theta, z, z, np.full(theta.size, 1e-8), 1, LR)
    res["eps_outside_root"] = np.allclose(th1 - theta, -LR / 2, rtol=1e-9, atol=0)
    # a constant gradient for ten steps: the same move every step
    th, m, v = theta, z, z
    for t in range(1, 11):
        th, m, v = adam_step(th, m, v, g, t, LR)
    res["constant_gradient"] = np.allclose(th - theta, -10 * LR * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)
    # worked by hand, one parameter: g = +1 then -1.  m_2 = 0.9 * 0.1 - 0.1 = -0.01,
    # v_2 = 0.999 * 0.001 + 0.001 = 0.001999 = 1 - 0.999^2, so m_hat = -0.01 / 0.19 = -1/19
    # and v_hat = 1: the second step moves by +lr / (19 (1 + eps))
    one = np.zeros(theta.size)
    one[0] = 1.0
    a, ma, va = adam_step(theta, z, z, one, 1, LR)
    b, _, _ = adam_step(a, ma, va, -one, 2, LR)
    res["two_steps_by_hand"] = (abs((a[0] - theta[0]) - (-LR / (1 + 1e-8))) <= 1e-15 and
                                abs((b[0] - a[0]) - LR / (19 * (1 + 1e-8))) <= 1e-15)
    # L2 decay on the weight matrices only: with g = 0 a weight moves against its sign
    # by lr |wd w| / (|wd w| + eps) and a bias does not move
    theta_b = theta.copy()
    for k in (1, 3, 5, 7):
        theta_b[_bias_slice(k)] = rng.standard_normal(_bias_slice(k).stop - _bias_slice(k).start)
    th1, _, _ = adam_step(theta_b, z, z, z, 1, LR, weight_decay=0.01)
    w = mlp.weight_mask() > 0
    d = 0.01 * np.abs(theta_b[w])
    res["decay_weights"] = np.allclose(th1[w] - theta_b[w], -LR * np.sign(theta_b[w]) * d / (d + 1e-8),
                                       rtol=1e-12, atol=1e-18)
    res["no_decay_biases"] = np.array_equal(th1[~w], theta_b[~w])
    return res


def test_adam_pins():
    res = _adam_pins(mlp.adam_step)
    assert all(res.values()), res


def test_weight_mask_covers_the_matrices():
    w = mlp.weight_mask()
    assert int(w.sum()) == 256 * 36 + 256 * 256 * 2 + 128 * 256
    assert w.size == mlp.N_PARAMS


ADAM_MUTANTS = {
    "no_bias_correction": ("m_hat = m / (1.0 - beta1 ** t)", "m_hat = m"),
    "no_second_correction": ("v_hat = v / (1.0 - beta2 ** t)", "v_hat = v"),
    "eps_inside_root": ("(np.sqrt(v_hat) + eps)", "np.sqrt(v_hat + eps)"),
    "decay_on_biases": ("weight_decay * weight_mask() * theta", "weight_decay * theta"),
    "decoupled_decay": ("g = np.asarray(grad, dtype=np.float64) + weight_decay * weight_mask() * theta",
                        "g = np.asarray(grad, dtype=np.float64)"),
    "correction_exponent": ("1.0 - beta1 ** t", "1.0 - beta1 ** (t + 1)"),
}


def _mutant_module(old, new):
    import inspect
    import types
    src = inspect.getsource(mlp)
    assert old in src, old
    mod = types.ModuleType("mlp_mutant")
    exec(compile(src.replace(old, new), "mlp_mutant", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(ADAM_MUTANTS))
def test_adam_mutants_fail_a_pin(name):
    old, new = ADAM_MUTANTS[name]
    mod = _mutant_module(old, new)
    res = _adam_pins(mod.adam_step)
    assert not all(res.values()), f"mutant {name} passes every Adam pin"


# ---------------------------------------------------------------- BF16 rounding points

def _integer_net(rng, batch):
    """Weights in {-1, 0, 1}, integer inputs and biases: every value of the network is a
    small integer, exactly representable in bfloat16, so rounding must change nothing."""
    parts = []
    for s in mlp.SHAPES:
        if len(s) == 2:
            parts.append(rng.integers(-1, 2, s) * (rng.random(s) < 0.02))
        else:
            parts.append(rng.integers(-2, 3, s))
    theta = mlp.pack(parts).astype(np.float64)
    x = rng.integers(-3, 4, (batch, 36)).astype(np.float64)
    return theta, x


def test_bf16_forward_equals_exact_on_representable_values():
    rng = np.random.default_rng(21)
    theta, x = _integer_net(rng, 6)
    y, _ = mlp.forward(theta, x)
    yb, (xb, a1, a2, a3), _ = mlp.forward_bf16(theta, x)
    assert np.abs(y).max() < 256 and np.abs(y).max() > 0
    assert np.array_equal(yb, y)


def test_bf16_forward_rounds_each_hidden_activation():
    """One path through the network, worked by hand: x = 257 reaches unit 0 of layer 1
    with weight 1; 257 needs nine significant bits and rounds (tie to even) to 256, which
    layers 2 and 3 pass on with weight 1 and a bias of 1 each: 257 rounds to 256 again
    at both; the output unit adds 1 with no rounding: 257.  Unrounded the path gives 260."""
    W1, b1, W2, b2, W3, b3, W4, b4 = [np.zeros(s) for s in mlp.SHAPES]
    W1[0, 0] = 1.0
    W2[0, 0] = W3[0, 0] = W4[0, 0] = 1.0
    b2[0] = b3[0] = b4[0] = 1.0
    theta = mlp.pack([W1, b1, W2, b2, W3, b3, W4, b4])
    x = np.zeros((1, 36))
    x[0, 0] = 257.0
    yb, (xb, a1, a2, a3), _ = mlp.forward_bf16(theta, x)
    assert xb[0, 0] == 256.0 and a1[0, 0] == 256.0 and a2[0, 0] == 256.0 and a3[0, 0] == 256.0
    assert yb[0, 0] == 257.0
    assert mlp.forward(theta, x)[0][0, 0] == 260.0


def test_bf16_gradient_equals_exact_on_representable_values():
    rng = np.random.default_rng(22)
    theta, x = _integer_net(rng, 1)
    y, _ = mlp.forward(theta, x)
    # batch 1, n = 128: dY = (y - t) / 64 is exact in bfloat16 for |y - t| < 256 integers
    t = y - rng.integers(-3, 4, y.shape)
    l, g = mlp.loss_and_grad(theta, x, t)
    lb, gb, sc = mlp.loss_and_grad_bf16(theta, x, t)
    assert l == lb and np.array_equal(g, gb)
    # batch 1: every weight gradient is one term, so its scale is its magnitude
    w = mlp.weight_mask() > 0
    assert np.array_equal(sc[w], np.abs(gb[w]))
    assert np.all(sc >= np.abs(gb))

