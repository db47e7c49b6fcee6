"""The crop-replay machinery on the host: crops of an oracle state, replayed by the oracle,
reproduce a whole-raster oracle run on the kept cells (all four sides and a free outlet
interval included) to float64 rounding -- the replayed dt is recovered from the time
levels, (t + dt) - t, which may differ from dt in the last bit."""
import numpy as np

from crop_replay import CROP, compare_crops, crop_bc, pick_crops
from paper_2406_14933_gb300 import inputs


def test_crops_reproduce_the_whole_raster(orc):
    sc = inputs.tiny(96, 110, seed=5, bc=(1, 0, 1, 1), rain_mm_h=30.0, smooth=True)
    sc.free_range = ((0, 0), (0, 0), (30, 61), (0, 0))       # S side free on columns 30..60 only
    p = orc.from_scenario(sc)
    m = p.mass(sc.h0)
    res = p.run(m, sc.v1_0, sc.v2_0, 0.0, 1e9, max_steps=5)
    t0 = res["t"]
    s0 = (res["m"].reshape(96, 110), res["v1"].reshape(96, 110), res["v2"].reshape(96, 110))
    ts, st = [], s0
    cur = dict(m=res["m"], v1=res["v1"], v2=res["v2"], t=t0)
    for _ in range(3):
        cur = p.run(cur["m"], cur["v1"], cur["v2"], cur["t"], 1e9, max_steps=1)
        ts.append(cur["t"])
    s1 = (cur["m"].reshape(96, 110), cur["v1"].reshape(96, 110), cur["v2"].reshape(96, 110))
    crops = pick_crops(sc, np.random.default_rng(0), 8,
                       extra=[(0, 0), (0, 110 - CROP), (96 - CROP, 0), (96 - CROP, 110 - CROP), (0, 20)])
    eh, eq, n = compare_crops(orc, sc, crops, t0, ts, s0, s1)
    assert n > 0
    assert eh <= 1e-13 and eq <= 1e-13


def test_crop_boundary_conditions():
    sc = inputs.tiny(96, 110, seed=5, bc=(1, 0, 1, 1))
    sc.free_range = ((0, 0), (0, 0), (30, 61), (0, 0))
    bc, fr, margin = crop_bc(sc, 0, 20)
    assert bc == (0, 0, 1, 0) and fr[2] == (10, 41) and margin == [3, 3, 0, 3]
    bc, fr, margin = crop_bc(sc, 0, 62)                      # outlet interval outside the crop
    assert bc[2] == 0 and margin[2] == 0
    bc, fr, margin = crop_bc(sc, 96 - CROP, 110 - CROP)       # N and E sides: free, wall
    assert bc == (0, 0, 0, 1) and fr[3] == (0, 0) and margin == [3, 0, 3, 0]
