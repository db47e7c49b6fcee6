"""The allocation-free scan (asx_state_scan_noalloc) against the allocating path.

Callers that may not allocate device memory (a runtime that owns every buffer, a library
that only lends pointers) get the storage / wave-speed scan of a state they hold, with
the library's scratch in a fixed device array.  This file is collected last so that a run
stopping at its first failure has already run every other test; it passes alone and after
the others.
"""
import numpy as np
import pytest

from paper_2406_14933_gb300 import inputs

pytestmark = pytest.mark.gpu


def _state_on_device(R, torch):
    """The raster's state through the existing entry point, copied to dense device tensors."""
    from paper_2406_14933_gb300 import asx as A
    sh = (R.sc.rows, R.sc.cols)
    mh, ml, v1, v2 = (torch.empty(sh, dtype=torch.float32, device="cuda") for _ in range(4))
    A.asx_get_state(R.handle, mh.data_ptr(), ml.data_ptr(), v1.data_ptr(), v2.data_ptr(), A.ASX_PTR_DEVICE)
    return mh, ml, v1, v2


@pytest.mark.parametrize("rows,cols", [(24, 40), (301, 517)])
def test_noalloc_scan_matches_existing_entry_point(asx, rows, cols):
    import torch
    from paper_2406_14933_gb300 import asx as A
    from paper_2406_14933_gb300.raster import Raster
    sc = inputs.tiny(rows, cols, seed=rows + cols, bc=(1, 1, 0, 0), rain_mm_h=30.0, smooth=True)
    R = Raster(sc)
    R.step(7)
    mh, ml, v1, v2 = _state_on_device(R, torch)
    theta = torch.from_numpy(np.ascontiguousarray(sc.theta)).cuda()
    storage = torch.zeros(1, dtype=torch.float64, device="cuda")
    cmax = torch.zeros(1, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ref_storage = R.ledger().storage                       # existing entry point
    # the wave speed of the same state, from the state the existing entry point returned
    h = (mh.double() / theta.double()).cpu().numpy()
    ref_cmax = (np.hypot(v1.double().cpu().numpy(), v2.double().cpu().numpy()) + np.sqrt(sc.g * h)).max()
    for _ in range(2):                                     # two calls in a row share the scratch
        storage.zero_()
        cmax.zero_()
        A.asx_state_scan_noalloc(rows, cols, cols, sc.l, sc.g, mh, ml, v1, v2, theta, storage, cmax,
                                 stream)
        torch.cuda.synchronize()
        assert float(storage[0]) == pytest.approx(ref_storage, rel=1e-12)
        assert float(cmax[0]) == pytest.approx(ref_cmax, rel=1e-6)
    R.close()


def test_noalloc_scan_rejects_oversize(asx):
    from paper_2406_14933_gb300 import asx as A
    with pytest.raises(A.AsxError) as e:
        # 8192 x 8193 cells exceeds the scratch's 67,108,864-cell limit (checked before
        # any pointer is touched)
        A.asx_state_scan_noalloc(8192, 8193, 8193, 1.0, 9.81, 1, 1, 1, 1, 1, 1, 1, None)
    assert e.value.status == A.ASX_EINVAL
    for g in (float("inf"), float("nan"), 0.0):
        with pytest.raises(A.AsxError) as e:
            A.asx_state_scan_noalloc(8, 8, 8, 1.0, g, 1, 1, 1, 1, 1, 1, 1, None)
        assert e.value.status == A.ASX_EINVAL


def test_noalloc_scan_pitched_state(asx):
    """A state held in wider buffers (row pitch > cols): every field, theta included,
    is a column slice of a device tensor with extra columns that hold other values, and
    the scan matches the dense result, twice in a row."""
    import torch
    from paper_2406_14933_gb300 import asx as A
    from paper_2406_14933_gb300.raster import Raster
    rows, cols, pitch = 97, 133, 160
    sc = inputs.tiny(rows, cols, seed=5, bc=(1, 0, 1, 0), rain_mm_h=50.0, smooth=True)
    R = Raster(sc)
    R.step(5)
    dense = _state_on_device(R, torch)
    theta = torch.from_numpy(np.ascontiguousarray(sc.theta)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    wide = []
    for t in (*dense, theta):
        w = torch.full((rows, pitch), 1.0e3, dtype=torch.float32, device="cuda")   # junk outside the slice
        w[:, :cols] = t
        wide.append(w)
    out = []
    for fields, p in ((dense + (theta,), cols), (tuple(wide), pitch)):
        st = torch.zeros(1, dtype=torch.float64, device="cuda")
        cm = torch.zeros(1, dtype=torch.float32, device="cuda")
        A.asx_state_scan_noalloc(rows, cols, p, sc.l, sc.g, *fields, st, cm, stream)
        torch.cuda.synchronize()
        out.append((float(st[0]), float(cm[0])))
    A.asx_state_scan_noalloc(rows, cols, pitch, sc.l, sc.g, *wide, st, cm, stream)
    torch.cuda.synchronize()
    assert out[0] == out[1] == (float(st[0]), float(cm[0]))
    assert out[0][0] == pytest.approx(R.ledger().storage, rel=1e-12)
    R.close()
