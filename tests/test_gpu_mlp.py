"""The surrogate MLP on the tensor cores against the FP64 reference.

The kernels store BF16 operands (inputs, weights, hidden activations, back-propagated
gradients) and accumulate in FP32.  The oracle's BF16 mirror (`forward_bf16`,
`loss_and_grad_bf16`) rounds the same operands at the same points and forms every sum
exactly, so the two differ only by the FP32 accumulation order (a relative 1e-6 of a
sum's magnitude) and, where an FP32 sum lies within that of a bfloat16 rounding boundary
or of zero, by one bfloat16 unit (at most 2^-7 of the value) of one stored operand.  So
every output element is held to 2^-7 of its own magnitude sum s (the sum of the absolute
values of the terms that form it: sum_k |W_jk| a_k + |b_j| for an output, sum_m |dZ| |A|
for a weight gradient, sum_m |dZ| for a bias gradient), plus, for gradients, 2^-6 where a
rounding flip upstream spreads through one more layer.  A wrong column, bias, mask or
rounding point errs by a sizeable fraction of s.
"""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def _setup(asx, batch, seed=0, max_batch=None):
    from paper_2406_14933_gb300 import asx as A
    rng = np.random.default_rng(seed)
    theta = ref.init_params(rng)
    theta[ref.N_PARAMS - 128:] = rng.standard_normal(128) * 0.1       # non-zero output bias
    theta = ref.to_bf16(theta)
    x = ref.to_bf16(rng.standard_normal((batch, 36)))
    t = rng.standard_normal((batch, 128)) * 0.5
    p = A.asx_mlp_create(max_batch=max_batch or max(batch, 128))
    A.asx_mlp_set_params(p, np.ascontiguousarray(theta, np.float32))
    return A, p, theta, x, t


def _output_scale(theta, x):
    """Per output element: sum_k |W4_jk| a3_k + |b4_j| of the BF16 mirror."""
    _, (_, _, _, a3), Wb = ref.forward_bf16(theta, x)
    b4 = ref.unpack(theta)[7]
    return a3 @ np.abs(Wb[3]).T + np.abs(b4)


def _check_forward(y, theta, x):
    yr, _, _ = ref.forward_bf16(theta, x)
    s = _output_scale(theta, x)
    d = np.abs(np.asarray(y, np.float64) - yr)
    worst = float((d / s).max())
    assert np.all(d <= 2.0 ** -7 * s), worst
    # rounding flips are rare: the bulk of the elements agrees to the FP32 accumulation
    # order (a wrong rounding mode or a systematic offset would move these quantiles)
    r = d / s
    assert float(np.median(r)) <= 2.0 ** -18 and float(np.quantile(r, 0.99)) <= 2.0 ** -12, worst


@pytest.mark.parametrize("batch", [1, 77, 128, 129, 300, 1024])
def test_forward_matches_reference(asx, batch):
    A, p, theta, x, t = _setup(asx, batch)
    y = np.empty((batch, 128), np.float32)
    A.asx_mlp_forward(p, batch, np.ascontiguousarray(x, np.float32), y)
    _check_forward(y, theta, x)
    back = np.empty(ref.N_PARAMS, np.float32)
    A.asx_mlp_get_params(p, back)
    assert np.array_equal(back, theta.astype(np.float32))
    A.asx_mlp_destroy(p)


@pytest.mark.parametrize("batch", [1, 129, 40000, 65536])
def test_fused_forward_matches_reference_device(asx, batch):
    """The fused persistent kernel on device-resident queries, the whole batch in one
    launch (at 40,000 and 65,536 queries each CTA loops over several 128-query tiles),
    element by element against the oracle's BF16 mirror."""
    import torch
    A, p, theta, x, t = _setup(asx, batch, seed=batch, max_batch=1024)
    xd = torch.tensor(np.ascontiguousarray(x, np.float32), device="cuda")
    yd = torch.full((batch, 128), float("nan"), dtype=torch.float32, device="cuda")
    A.asx_mlp_forward(p, batch, xd.data_ptr(), yd.data_ptr(), A.ASX_PTR_DEVICE)
    _check_forward(yd.cpu().numpy(), theta, x)
    A.asx_mlp_destroy(p)


@pytest.mark.parametrize("batch", [1, 64, 256, 1000])
def test_gradients_match_reference(asx, batch):
    A, p, theta, x, t = _setup(asx, batch, seed=batch)
    g = np.empty(ref.N_PARAMS, np.float32)
    xs, ts = np.ascontiguousarray(x, np.float32), np.ascontiguousarray(t, np.float32)
    loss = A.asx_mlp_gradients(p, batch, xs, ts, g)
    lr_, gr, sc = ref.loss_and_grad_bf16(theta, x, t)
    assert loss == pytest.approx(lr_, rel=1e-4)
    d = np.abs(g.astype(np.float64) - gr)
    o = 0
    for k, s in enumerate(ref.SHAPES):
        n = int(np.prod(s))
        sl = slice(o, o + n)
        assert np.all(d[sl] <= 2.0 ** -6 * sc[sl] + 1e-30), (k, float((d[sl] / (sc[sl] + 1e-300)).max()))
        o += n
    # the gradient pass is deterministic (fixed-order sums): a second call gives the same bits
    g2 = np.empty_like(g)
    A.asx_mlp_gradients(p, batch, xs, ts, g2)
    assert np.array_equal(g, g2)
    A.asx_mlp_destroy(p)


@pytest.mark.parametrize("batches", [[256] * 5, [64, 100, 64, 100, 64, 100, 64]], ids=["fixed", "alternating"])
@pytest.mark.parametrize("wd", [0.0, 1e-2])
def test_adam_step_matches_reference(asx, wd, batches):
    """Adam steps of asx_mlp_train_step (the first step at a batch size runs its kernels
    eagerly, the second captures them in a CUDA graph, later ones replay it with new
    scalars; the alternating schedule keeps a graph per batch size), each parameter
    update against the oracle's
    FP64 Adam step from the same parameters, moments and gradient (the gradient read back
    with asx_mlp_gradients, which the train step computes bit for bit the same).  FP32
    arithmetic leaves each updated parameter within a few units in its last place of the
    FP64 update, |theta_gpu - theta_ref| <= 4 ulp(theta_ref) + 1e-5 |d theta|, plus the
    first-order effect of rounding the decayed gradient g' = g + wd theta in FP32
    (|delta g'| <= 2^-22 (|g| + wd |theta|), carried by the moments): where g' nearly
    cancels, Adam's m_hat / (sqrt(v_hat) + eps) turns it into
    lr (dm / (sqrt(v_hat) + eps) + |m_hat| dv / (2 sqrt(v_hat) (sqrt(v_hat) + eps)^2)).
    After the steps the forward pass uses the refreshed BF16 copies of the new weights."""
    from paper_2406_14933_gb300 import asx as A
    rng = np.random.default_rng(17)
    theta = ref.init_params(rng).astype(np.float32)
    p = A.asx_mlp_create(max_batch=max(batches))
    A.asx_mlp_set_params(p, theta)
    m = np.zeros(ref.N_PARAMS)
    v = np.zeros(ref.N_PARAMS)
    cur = theta.astype(np.float64)
    lr = 1e-3
    wmask = ref.weight_mask()
    dmax = np.zeros(ref.N_PARAMS)       # largest rounding of g' so far, per parameter
    gmax = np.zeros(ref.N_PARAMS)       # largest |g'| so far
    for step, batch in enumerate(batches, 1):
        x = rng.uniform(-1, 1, (batch, 36)).astype(np.float32)
        t = rng.uniform(0, 1, (batch, 128)).astype(np.float32)
        g = np.empty(ref.N_PARAMS, np.float32)
        A.asx_mlp_gradients(p, batch, x, t, g)
        A.asx_mlp_train_step(p, batch, x, t, lr, wd)
        new = np.empty(ref.N_PARAMS, np.float32)
        A.asx_mlp_get_params(p, new)
        want, m, v = ref.adam_step(cur, m, v, g.astype(np.float64), step, lr, weight_decay=wd)
        gd = g.astype(np.float64) + wd * wmask * cur
        dmax = np.maximum(dmax, 2.0 ** -22 * (np.abs(g) + wd * wmask * np.abs(cur)))
        gmax = np.maximum(gmax, np.abs(gd))
        mh, vh = np.abs(m) / (1 - 0.9 ** step), v / (1 - 0.999 ** step)
        sv = np.sqrt(vh)
        dv = 2.0 * gmax * dmax
        sens = lr * (dmax / (sv + 1e-8) + mh * dv / (2.0 * np.maximum(sv, 1e-30) * (sv + 1e-8) ** 2))
        d = np.abs(new.astype(np.float64) - want)
        tol = 4.0 * np.spacing(np.abs(want).astype(np.float32)).astype(np.float64) + 1e-5 * np.abs(want - cur) + sens
        assert np.all(d <= tol), (step, float((d / tol).max()))
        cur = new.astype(np.float64)
    xq = rng.uniform(-1, 1, (300, 36)).astype(np.float32)
    y = np.empty((300, 128), np.float32)
    A.asx_mlp_forward(p, 300, xq, y)
    _check_forward(y, cur, xq)
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

