"""Host-side pieces of the surrogate: the input encoding and the scenario draws."""
import math

import numpy as np
import pytest

from paper_2406_14933_gb300 import surrogate as S
from paper_2406_14933_gb300.inputs import MM_PER_H, constant_rain, ensemble_member, member_params, triangular_rain


def test_hyetograph_bins_integrate_to_rain_depth():
    # block storm shorter than the window: bins sum to rate x duration
    rt, rr = constant_rain(90.0, 1500.0)
    h = S.hyetograph(rt, rr)
    assert h.sum() * (3600.0 / 32) == pytest.approx(90.0 * MM_PER_H * 1500.0, rel=1e-12)
    # 1500 s = 13 full bins of 112.5 s and a third of the 14th
    assert np.all(h[:13] == pytest.approx(90.0 * MM_PER_H))
    assert h[13] == pytest.approx(90.0 * MM_PER_H * (1500.0 - 13 * 112.5) / 112.5)
    assert np.all(h[14:] == 0.0)
    # triangle (Appendix C shape): half base times height, and the bin containing the peak
    rt, rr = triangular_rain(3000.0, 1000.0, 120.0)
    h = S.hyetograph(rt, rr)
    assert h.sum() * 112.5 == pytest.approx(0.5 * 3000.0 * 120.0 * MM_PER_H, rel=1e-12)
    # bin 8 = [900, 1012.5] holds the peak: (int_900^1000 0.12 t dt + int_0^12.5 (120 - 0.06 u) du) / 112.5
    assert h[8] == pytest.approx(114.625 * MM_PER_H, rel=1e-12)
    # rain beyond the window is cut off
    rt, rr = constant_rain(60.0, 5000.0)
    assert S.hyetograph(rt, rr).sum() * 112.5 == pytest.approx(60.0 * MM_PER_H * 3600.0, rel=1e-12)


def test_cumulative_rain_is_piecewise_quadratic():
    rt, rr = np.array([0.0, 100.0, 300.0]), np.array([0.0, 2.0, 0.0])
    t = np.array([0.0, 50.0, 100.0, 200.0, 300.0, 400.0])
    # integral of the tent by hand
    exp = np.array([0.0, 0.5 * 50 * 1.0, 100.0, 100.0 + 0.5 * (2.0 + 1.0) * 100.0, 300.0, 300.0])
    assert np.allclose(S.cumulative_rain(rt, rr, t), exp, rtol=0, atol=1e-12)


def test_query_features_match_full_scenarios():
    Xq, Sq = S.query_features(S.QUERY_SEED0, 5, n=48, l=8.0, start=3)
    for i in range(5):
        sc = S.scenario(S.QUERY_SEED0, 3 + i, n=48, l=8.0)
        assert np.array_equal(S.features(sc), Xq[i])
        assert S.discharge_scale(sc) == pytest.approx(Sq[i], rel=1e-12)
        assert sc.sample_dt == 50.0 and sc.t_end == 6400.0
    x = Xq[0]
    assert np.all(np.abs(x[:4]) <= 1.0) and np.all(x[4:] >= 0.0) and np.all(x[4:] <= 1.0)


def test_member_params_are_the_members_draws():
    for s in range(4):
        d = member_params(s, 5_000_000, n_override=40)
        m = ensemble_member(s, 5_000_000, n_override=40).meta
        for k in ("slope", "cover", "theta", "alpha_p", "rain_mm_h", "rain_s"):
            assert d[k] == m[k]


def test_cover_patches_keep_their_physical_size():
    a = S.scenario(S.TRAIN_SEED0, 7, n=64, l=8.0)
    veg = a.theta < 1.0
    assert abs(veg.mean() - a.meta["cover"]) < 2.0 / veg.size + 1e-9
    assert S.COVER_CORR_M / 8.0 == 2.0


def test_init_params_layout():
    p = S.init_params(np.random.default_rng(0))
    assert p.size == S.N_PARAMS == 173952
    o = 0
    for out, inp in S.LAYERS:
        w = p[o:o + out * inp]
        assert abs(w.std() - math.sqrt(2.0 / inp)) < 0.05 * math.sqrt(2.0 / inp)
        o += out * inp
        assert np.all(p[o:o + out] == 0.0)
        o += out
