"""The bounds-checked debug build: the step kernel compiled with ASX_BOUNDS_CHECK checks every
shared-memory ring index and global store of its tiles and reports a violation as
ASX_EBOUNDS (the stand-in for a memory checker, which this pool does not offer).  Raster
shapes that exercise the tile layout (several tiles, an overlapping last strip and row
block, a single strip, tall and wide rasters, land-cover classes) run without a violation,
and agree with the ordinary build (the checks change no arithmetic; the code generator may
contract the momentum sums differently, so the comparison allows 1e-5)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json
import numpy as np
from paper_2406_14933_gb300 import inputs
from paper_2406_14933_gb300.raster import Raster
out = []
for rows, cols, seed, classes in [(200, 700, 91, False), (36, 150, 3, False), (35, 137, 4, False),
                                  (300, 133, 5, True), (67, 1000, 6, True)]:
    sc = inputs.tiny(rows, cols, seed, bc=(inputs.FLUX, inputs.FREE, inputs.WALL, inputs.FREE), rain_mm_h=30.0)
    sc.bc_q = (0.01, 0.0, 0.0, 0.0)
    if classes:
        rng = np.random.default_rng(seed)
        sc.cls = rng.integers(0, 3, size=(rows, cols)).astype(np.uint8)
        sc.class_theta = np.array([0.9, 0.97, 1.0], np.float32)
        sc.class_alpha_p = np.array([80.0, 40.0, 0.0], np.float32)
        sc.class_alpha_s = np.array([0.00709, 0.00709, 0.00709], np.float32)
    R = Raster(sc)
    R.step(40)
    m, v1, v2 = R.mass64()
    led = R.ledger()
    R.close()
    out.append(dict(shape=[rows, cols], m=float(m.sum()), v=float(np.abs(v1).sum() + np.abs(v2).sum()),
                    defect=led.defect_rel))
print(json.dumps(out))
'''


def _run(lib):
    env = dict(os.environ, ASX_STEP_KERNEL="strip")
    env.pop("ASX_LIB", None)
    if lib:
        env["ASX_LIB"] = lib
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_finds_no_violation(asx):
    from paper_2406_14933_gb300 import build
    checked = _run(build.build_checked())
    plain = _run(None)
    for c, p in zip(checked, plain):
        print(f"[bounds] {c['shape']}: mass {c['m']:.9g} vs {p['m']:.9g}, defect {c['defect']:.1e}")
        assert c["m"] == pytest.approx(p["m"], rel=1e-5)
        assert c["v"] == pytest.approx(p["v"], rel=1e-5)
        assert c["defect"] <= 1e-10
