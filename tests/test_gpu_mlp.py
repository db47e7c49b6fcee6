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


@pytest.mark.parametrize("batch", [1, 127, 128, 129, 1000, 40000])
def test_fused_forward_matches_layered(asx, batch, monkeypatch):
    """The fused four-layer kernel against the layer-by-layer GEMMs: the same BF16
    rounding points and the same FP32 accumulation order, device pointers (the whole
    batch in one launch, beyond the handle's max_batch) and host pointers."""
    import torch

    from paper_2406_14933_gb300 import asx as A
    rng = np.random.default_rng(batch)
    theta = ref.init_params(rng).astype(np.float32)
    theta[ref.N_PARAMS - 128:] = rng.standard_normal(128) * 0.1       # non-zero output bias
    x = rng.standard_normal((batch, 36)).astype(np.float32)
    p = A.asx_mlp_create(max_batch=1024)
    A.asx_mlp_set_params(p, theta)
    xd = torch.tensor(x, device="cuda")
    yf = torch.empty((batch, 128), dtype=torch.float32, device="cuda")
    A.asx_mlp_forward(p, batch, xd.data_ptr(), yf.data_ptr(), A.ASX_PTR_DEVICE)
    yh = np.empty((batch, 128), np.float32)
    A.asx_mlp_forward(p, batch, x, yh)                                   # host pointers
    monkeypatch.setenv("ASX_MLP_FUSED", "0")
    yl = np.empty((batch, 128), np.float32)
    A.asx_mlp_forward(p, batch, x, yl)
    monkeypatch.delenv("ASX_MLP_FUSED")
    yf = yf.cpu().numpy()
    scale = float(np.abs(yl).max())
    assert np.abs(yf - yl).max() <= 1e-5 * scale
    assert np.array_equal(yf, yh)
    # misaligned device pointers take the staged path
    xm = torch.empty(batch * 36 + 1, dtype=torch.float32, device="cuda")
    xm[1:] = xd.reshape(-1)
    ym = torch.empty(batch * 128 + 1, dtype=torch.float32, device="cuda")
    A.asx_mlp_forward(p, batch, xm.data_ptr() + 4, ym.data_ptr() + 4, A.ASX_PTR_DEVICE)
    assert np.array_equal(ym[1:].cpu().numpy().reshape(batch, 128), yf)
    A.asx_mlp_destroy(p)


def test_fused_forward_follows_training(asx):
    """After Adam steps the fused kernel uses the updated weights (its weight image is
    rebuilt), matching the layered pass."""
    import os
    from paper_2406_14933_gb300 import asx as A
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (512, 36)).astype(np.float32)
    t = rng.uniform(0, 1, (512, 128)).astype(np.float32)
    p = A.asx_mlp_create(max_batch=512)
    A.asx_mlp_set_params(p, ref.init_params(rng).astype(np.float32))
    y0 = np.empty((512, 128), np.float32)
    A.asx_mlp_forward(p, 512, x, y0)
    for _ in range(5):
        A.asx_mlp_train_step(p, 512, x, t, 1e-3)
    y1 = np.empty((512, 128), np.float32)
    A.asx_mlp_forward(p, 512, x, y1)
    os.environ["ASX_MLP_FUSED"] = "0"
    try:
        yl = np.empty((512, 128), np.float32)
        A.asx_mlp_forward(p, 512, x, yl)
    finally:
        del os.environ["ASX_MLP_FUSED"]
    assert not np.array_equal(y0, y1)
    assert np.abs(y1 - yl).max() <= 1e-5 * float(np.abs(yl).max())
    A.asx_mlp_destroy(p)
