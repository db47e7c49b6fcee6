"""The strip kernel's mass increments are the scalar code's, bit for bit.

Each edge's mass increment is evaluated twice wherever it joins two lanes of a tile, two
tiles or a tile and the frame, and once more by the gather kernel; the water budget
closes only if every evaluation gives the same bits.  From the same flowing state, one
step of the strip kernel and one of the gather kernel must therefore give the same cell
masses up to the order of the compensated additions (float64 rounding, ~1e-15 of a cell's
mass), while a single increment that differs in its last bit shows at ~1e-9 (a float32
rounding of the increment).  Checked with per-cell porosity, with land-cover classes and
with the optional terms compiled in, on a raster of several tiles whose last strip and
row block overlap the previous ones, with a given-flux side, free sides and rain; and the
strip kernel's budget over 300 steps, far below the stated 1e-10.
"""
import numpy as np
import pytest

from paper_2406_14933_gb300 import asx as A
from paper_2406_14933_gb300 import inputs

pytestmark = pytest.mark.gpu


def _scenario(mode):
    sc = inputs.tiny(200, 700, 91, bc=(inputs.FLUX, inputs.FREE, inputs.WALL, inputs.FREE), relief=0.5,
                     rain_mm_h=40.0)
    sc.bc_q = (0.02, 0.0, 0.0, 0.0)
    if mode == "classes":
        rng = np.random.default_rng(92)
        sc.cls = rng.integers(0, 3, size=(sc.rows, sc.cols)).astype(np.uint8)
        sc.class_theta = np.array([0.9, 0.97, 1.0], np.float32)
        sc.class_alpha_p = np.array([80.0, 40.0, 0.0], np.float32)
        sc.class_alpha_s = np.array([0.00709, 0.00709, 0.00709], np.float32)
    if mode == "optional":
        sc.viscosity = True
        sc.tau = 0.01
    return sc


@pytest.mark.parametrize("mode", ["theta", "classes", "optional"])
def test_strip_step_equals_gather_step(asx, monkeypatch, mode):
    from paper_2406_14933_gb300.raster import Raster
    sc = _scenario(mode)
    monkeypatch.setenv("ASX_STEP_KERNEL", "gather")
    R = Raster(sc)
    R.step(10)
    state = [np.ascontiguousarray(x) for x in R.state()]
    t, _, step = R.clock()
    led = R.ledger()
    R.close()
    masses = {}
    for kernel in ("gather", "strip"):
        monkeypatch.setenv("ASX_STEP_KERNEL", kernel)
        R = Raster(sc)
        A.asx_set_state(R.handle, *state, A.ASX_PTR_HOST, t, step, led)
        R.step(1)
        masses[kernel] = R.mass64()[0]
        R.close()
    mg, ms = masses["gather"], masses["strip"]
    scale = np.maximum(np.abs(mg), 1e-6 * np.abs(mg).max())
    worst = float(np.max(np.abs(ms - mg) / scale))
    print(f"[consistency] {mode}: worst cell mass difference {worst:.2e} of the cell's mass")
    assert worst <= 1e-12


def test_strip_budget_closes_to_rounding(asx, monkeypatch):
    from paper_2406_14933_gb300.raster import Raster
    monkeypatch.setenv("ASX_STEP_KERNEL", "strip")
    R = Raster(_scenario("classes"))
    R.step(300)
    d = R.ledger().defect_rel
    R.close()
    print(f"[consistency] strip budget defect after 300 steps {d:.2e}")
    assert d <= 1e-12
