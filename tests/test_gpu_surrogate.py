"""The surrogate end to end on the GPU: the check kernel against numpy, and the gain test.

The gain test runs the whole pipeline on 64 x 64 members with 8 m edges (the 512 m
hillslope of the full-size workload at a coarser cell, cover patches of the same 16 m),
so that it finishes in about a minute: solver runs for training and held-out data,
training with the tensor-core kernels, inference, and the 1 % solver check.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_check_kernel_matches_numpy(asx):
    import torch

    from paper_2406_14933_gb300 import surrogate as S
    rng = np.random.default_rng(11)
    B, K = 300, 40
    y = rng.standard_normal((B, 128)).astype(np.float32)
    idx = np.sort(rng.choice(B, K, replace=False)).astype(np.int32)
    ref = y[idx] + rng.standard_normal((K, 128)).astype(np.float32) * rng.uniform(0.0, 0.1, (K, 1)).astype(np.float32)
    ref[3] = 0.0
    y[idx[3]] = 0.0                       # both zero: error 0
    ref[5] = 0.0                          # only the solver's row zero: error inf
    idx_bad = idx.copy()
    idx_bad[7] = B + 5                    # outside the batch: skipped, NaN
    yd = torch.tensor(y, device="cuda")
    m = S.Surrogate(max_batch=128)
    err, nrep = m.check(yd, idx_bad, ref, tol=0.05)
    out = yd.cpu().numpy()
    e_np = np.linalg.norm(y[idx].astype(np.float64) - ref, axis=1) / np.maximum(np.linalg.norm(ref.astype(np.float64), axis=1), 1e-300)
    e_np[3] = 0.0
    e_np[5] = np.inf
    for k in range(K):
        if k == 7:
            assert np.isnan(err[k])
            assert np.array_equal(out[idx[k]], y[idx[k]])
            continue
        if np.isfinite(e_np[k]):
            assert err[k] == pytest.approx(e_np[k], rel=1e-5, abs=1e-7)
        else:
            assert np.isinf(err[k])
        if e_np[k] > 0.05:
            assert np.array_equal(out[idx[k]], ref[k])
        else:
            assert np.array_equal(out[idx[k]], y[idx[k]])
    untouched = np.setdiff1d(np.arange(B), idx)
    assert np.array_equal(out[untouched], y[untouched])
    assert nrep == int(sum(1 for k in range(K) if k != 7 and e_np[k] > 0.05))
    m.close()


def test_surrogate_gain_over_solver(asx):
    """Trained on solver runs, the network reproduces held-out hydrographs within 5 %
    relative L2, does much better than the mean training hydrograph, and serves queries
    (with 1 % of them re-solved and checked) far faster than the solver alone."""
    from paper_2406_14933_gb300 import surrogate as S
    rep, model = S.pipeline(n=64, l=8.0, n_train=8192, n_held=512, n_queries=16384, epochs=200, batch=256,
                            workers=0, chunk=4096)
    h, sv = rep["held_out"], rep["serve"]
    assert h["mean"] <= 0.05 and h["aggregate"] <= 0.05, h
    assert h["mean_hydrograph_baseline"] >= 3.0 * h["mean"], h
    assert sv["checked"] == 164
    assert sv["checked_mean_rel_l2"] <= 0.08, sv
    assert sv["replaced"] <= 0.25 * sv["checked"], sv
    assert sv["gain"] >= 20.0, sv
    model.close()
