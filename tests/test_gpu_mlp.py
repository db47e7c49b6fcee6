"""The surrogate MLP on the tensor cores against the FP64 reference.

BF16 tolerance: weights and inputs are given already rounded to bfloat16, so the GPU
differs from float64 only by rounding each activation and each back-propagated gradient
to bfloat16 (unit roundoff 2^-9) and by FP32 accumulation: a relative error of ~1 % per
tensor after four layers is expected, 3 % is the bound held here.
"""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def _setup(asx, batch, seed=0):
    from paper_2406_14933_gb300 import asx as A
    rng = np.random.default_rng(seed)
    theta = ref.to_bf16(ref.init_params(rng))
    x = ref.to_bf16(rng.standard_normal((batch, 36)))
    t = rng.standard_normal((batch, 128)) * 0.5
    p = A.asx_mlp_create(max_batch=max(batch, 128))
    A.asx_mlp_set_params(p, np.ascontiguousarray(theta, np.float32))
    return A, p, theta, x, t


@pytest.mark.parametrize("batch", [1, 77, 128, 300, 1024])
def test_forward_matches_reference(asx, batch):
    A, p, theta, x, t = _setup(asx, batch)
    y = np.empty((batch, 128), np.float32)
    A.asx_mlp_forward(p, batch, np.ascontiguousarray(x, np.float32), y)
    yr, _ = ref.forward(theta, x)
    assert _rel(y, yr) <= 3e-2
    back = np.empty(ref.N_PARAMS, np.float32)
    A.asx_mlp_get_params(p, back)
    assert np.array_equal(back, theta.astype(np.float32))
    A.asx_mlp_destroy(p)


@pytest.mark.parametrize("batch", [64, 256, 1000])
def test_gradients_match_reference(asx, batch):
    A, p, theta, x, t = _setup(asx, batch, seed=batch)
    g = np.empty(ref.N_PARAMS, np.float32)
    loss = A.asx_mlp_gradients(p, batch, np.ascontiguousarray(x, np.float32), np.ascontiguousarray(t, np.float32), g)
    lr_, gr = ref.loss_and_grad(theta, x, t)
    assert loss == pytest.approx(lr_, rel=3e-2)
    o = 0
    for s in ref.SHAPES:
        n = int(np.prod(s))
        assert _rel(g[o:o + n], gr[o:o + n]) <= 3e-2, s
        o += n
    A.asx_mlp_destroy(p)


def test_adam_training_reduces_loss(asx):
    """Adam on a smooth synthetic regression: the training loss falls by 10x."""
    from paper_2406_14933_gb300 import asx as A
    rng = np.random.default_rng(5)
    n = 2048
    x = rng.uniform(-1, 1, (n, 36)).astype(np.float32)
    w = rng.standard_normal((36, 128)) / 6
    tt = np.tanh(x @ w).astype(np.float32)
    p = A.asx_mlp_create(max_batch=256)
    A.asx_mlp_set_params(p, np.ascontiguousarray(ref.init_params(rng), np.float32))
    first = None
    for it in range(300):
        i = rng.choice(n, 256, replace=False)
        loss = A.asx_mlp_train_step(p, 256, np.ascontiguousarray(x[i]), np.ascontiguousarray(tt[i]), 1e-3)
        if first is None:
            first = loss
    y = np.empty((n, 128), np.float32)
    A.asx_mlp_forward(p, n, x, y)
    final = float(np.mean((y - tt) ** 2))
    assert final < first / 10, (first, final)
    A.asx_mlp_destroy(p)
