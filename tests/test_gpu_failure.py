"""Failure detection on the GPU without a fault: a bounded wait that nothing completes runs
out, the kernel flags it, the host reports ASX_ETIMEOUT, and the context stays usable
(a raster created afterwards steps and closes its water budget)."""
import time

import pytest

from paper_2406_14933_gb300 import asx as A
from paper_2406_14933_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_is_reported(asx):
    from paper_2406_14933_gb300.raster import Raster
    t0 = time.perf_counter()
    st = A.asx_selftest_wait(0)
    dt = time.perf_counter() - t0
    print(f"[failure] bounded wait gave up after {dt:.2f} s with status {st}")
    assert st == A.ASX_ETIMEOUT
    assert dt < 10.0
    R = Raster(inputs.tiny(40, 300, 7, bc=(inputs.WALL, inputs.FREE, inputs.WALL, inputs.WALL), rain_mm_h=20.0))
    R.step(50)
    assert R.ledger().defect_rel <= 1e-10
    R.close()
