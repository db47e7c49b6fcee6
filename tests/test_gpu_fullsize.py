"""Parity at full size, in the launch configuration the bench times.

The 4096 x 4096 carved catchment (the bench workload: strip kernel, 32-row tiles, land-cover
classes) and the 1024 x 1024 fractal basin run on the GPU into their storms.  Three more
steps follow, which the FP64 oracle replays at the GPU's time levels on 48 x 48 crops of
the GPU state: a cell's update only reads its six neighbours, so after three steps every
cell at least three rings inside a crop (or on a true raster side, with the raster's own
boundary condition there) depends on nothing outside it and can be compared one by one.
Crops start on even rows so that the odd-row offset of the hexagons is kept.

Tolerance: the stated one, relative L2 <= 1e-4 of depth and of discharge theta*h*v over
all compared cells (three float32 steps from the same state agree far closer; the bound
leaves room for the upwind and wet/dry decisions that rounding can flip).
"""
import numpy as np
import pytest

from crop_replay import CROP, K_STEPS, compare_crops, pick_crops
from paper_2406_14933_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(params=["strip", "gather"])
def variant(request, monkeypatch):
    monkeypatch.setenv("ASX_STEP_KERNEL", request.param)
    return request.param


def _run_and_compare(asx, orc, sc, t_stop, crops):
    from paper_2406_14933_gb300.raster import Raster
    R = Raster(sc)
    R.run_until(t_stop)
    t0 = R.clock()[0]
    m0, a0, b0 = R.mass64()
    ts = [R.step(1) for _ in range(K_STEPS)]
    m1, a1, b1 = R.mass64()
    R.close()
    return compare_crops(orc, sc, crops, t0, ts, (m0, a0, b0), (m1, a1, b1))


def test_catchment_4096_sampled_crops(asx, orc, variant):
    sc = inputs.carved_catchment()
    assert sc.rows == 4096 and sc.cols == 4096
    # the outlet lies on the south side: one crop holds it with the true free interval
    s_b, s_e = sc.free_range[2]                    # sides W, E, S, N = 0..3
    c_out = max(0, min(sc.cols - CROP, (s_b + s_e) // 2 - CROP // 2))
    crops = pick_crops(sc, np.random.default_rng(41), 16, extra=[(0, c_out)])
    eh, eq, n = _run_and_compare(asx, orc, sc, 2700.0, crops)
    print(f"[fullsize] catchment 4096^2 ({variant}): {n} cells, depth {eh:.2e}, discharge {eq:.2e}")
    assert n >= 15 * (CROP - 2 * K_STEPS) ** 2
    assert eh <= 1e-4 and eq <= 1e-4


def test_fractal_basin_1024_sampled_crops(asx, orc, variant):
    sc = inputs.fractal_basin()
    assert sc.rows == 1024 and sc.cols == 1024
    crops = pick_crops(sc, np.random.default_rng(43), 16, extra=[(0, 0), (sc.rows - CROP, sc.cols - CROP)])
    eh, eq, n = _run_and_compare(asx, orc, sc, 1800.0, crops)
    print(f"[fullsize] fractal basin 1024^2 ({variant}): {n} cells, depth {eh:.2e}, discharge {eq:.2e}")
    assert eh <= 1e-4 and eq <= 1e-4


def _rain_integral(rt, rr, t_end):
    """Integral of the piecewise-linear rain rate over [0, t_end], zero outside the table."""
    total = 0.0
    for k in range(len(rt) - 1):
        a, b = max(rt[k], 0.0), min(rt[k + 1], t_end)
        if b > a:
            s = (rr[k + 1] - rr[k]) / (rt[k + 1] - rt[k])
            total += 0.5 * (b - a) * (rr[k] + s * (a - rt[k]) + rr[k] + s * (b - rt[k]))
    return total


def test_catchment_4096_whole_storm(asx, orc, monkeypatch):
    """The bench workload through its whole 2 h storm from a dry start (~42,000 steps of the
    strip kernel): three steps shortly before t_end replayed by the oracle on crops (the
    outlet's among them, where the discharge is largest); at t_end the budget closes within
    the stated 1e-10 of the rain; the rain applied at the steps' right ends differs from
    the exact integral of the hyetograph by at most max|r'| dt_max t_end / 2 per unit
    area; and the hydrograph's samples add up to the outflow the ledger booked."""
    from paper_2406_14933_gb300.raster import Raster
    monkeypatch.setenv("ASX_STEP_KERNEL", "strip")
    sc = inputs.carved_catchment()
    s_b, s_e = sc.free_range[2]
    c_out = max(0, min(sc.cols - CROP, (s_b + s_e) // 2 - CROP // 2))
    crops = pick_crops(sc, np.random.default_rng(47), 8, extra=[(0, c_out)])
    R = Raster(sc)
    R.run_until(sc.t_end - 60.0)
    t0 = R.clock()[0]
    m0, a0, b0 = R.mass64()
    ts = [R.step(1) for _ in range(K_STEPS)]
    m1, a1, b1 = R.mass64()
    eh, eq, n = compare_crops(orc, sc, crops, t0, ts, (m0, a0, b0), (m1, a1, b1))
    R.run_until(sc.t_end)
    t, _, steps = R.clock()
    led = R.ledger()
    q = R.hydrograph()
    R.close()
    sigma = 1.5 * np.sqrt(3.0) * sc.l ** 2
    rt, rr = [float(x) for x in sc.rain_t], [float(x) for x in sc.rain_r]
    exact = sc.n * sigma * _rain_integral(rt, rr, sc.t_end)
    slope = max(abs(rr[k + 1] - rr[k]) / (rt[k + 1] - rt[k]) for k in range(len(rt) - 1))
    bound = sc.n * sigma * 0.5 * slope * sc.dt_max * sc.t_end
    print(f"[fullsize] whole storm: {steps} steps to t = {t:.0f} s; crops at t = {t0:.1f} s: {n} cells, "
          f"depth {eh:.2e}, discharge {eq:.2e}; defect {led.defect_rel:.2e}; rain {led.rain_in:.6e} m^3 "
          f"against {exact:.6e} exact; outflow {led.outflow:.4e} m^3, peak {q.max():.3f} m^3/s")
    assert t == sc.t_end and n >= 8 * (CROP - 2 * K_STEPS) ** 2
    assert eh <= 1e-4 and eq <= 1e-4
    assert led.defect_rel <= 1e-10
    assert abs(led.rain_in - exact) <= bound
    assert len(q) == round(sc.t_end / sc.sample_dt) and np.all(q >= 0.0)
    assert abs(q.sum() * sc.sample_dt - led.outflow) <= 1e-9 * led.outflow
