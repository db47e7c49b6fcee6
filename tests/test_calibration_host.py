"""The flume study's host logic (Sec. 4.3) on the CPU.

Oracle pins (oracle/calib.py against closed forms and hand-worked values):
  * delta_s, delta_p of a field linear in (alpha_s, alpha_p) are its two slopes; of
    alpha_s^2 + alpha_p^2 they are lo_s + hi_s and lo_p + hi_p exactly (the forward
    differences telescope: (a_{i+1}^2 - a_i^2) / d = a_i + a_{i+1});
  * chi of identical gauges is 0, of a constant offset the offset, of a hand example
    sqrt(2);
  * h_bar by hand on a three-cell row;
  * the pattern search finds the minimum of a quadratic inside the box, and the boundary
    point when the minimum lies outside it, and takes a hand-worked path on a separable
    quadratic; a search that drops the -step trial or the pattern move's (x - base) term
    fails one of these (planted in copies of the oracle).
Library against oracle: the same sensitivities, misfit and mean depth, and the batched
pattern search accepts exactly the oracle's sequence of base points.
Flume inputs: the inflow side's width against a brute-force count of its edges, the
inflow the oracle books against q_l, and a steady state with the artificial viscosity.
"""
import math
import os
import types

import numpy as np
import pytest

from paper_2406_14933_gb300 import calibration as C
from paper_2406_14933_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def oc():
    import oracle.calib as m
    return m


def _grid():
    a_s, a_p = C.grid_points(7, 5)
    return a_s, a_p, a_s[1] - a_s[0], a_p[1] - a_p[0]


# ----------------------------------------------------------------------------- oracle pins

def test_oracle_sensitivity_linear_field(oc):
    a_s, a_p, ds, dp = _grid()
    H = [[0.3 * s - 0.002 * p + 0.1 for p in a_p] for s in a_s]
    s, p = oc.sensitivity(H, ds, dp)
    assert s == pytest.approx(0.3, rel=1e-10) and p == pytest.approx(-0.002, rel=1e-10)


def test_oracle_sensitivity_quadratic_telescopes(oc):
    a_s, a_p, ds, dp = _grid()
    H = [[s * s + p * p for p in a_p] for s in a_s]
    s, p = oc.sensitivity(H, ds, dp)
    assert s == pytest.approx(a_s[0] + a_s[-1], rel=1e-9)
    assert p == pytest.approx(a_p[0] + a_p[-1], rel=1e-12)


def test_oracle_chi_by_hand(oc):
    assert oc.chi([[0.1, 0.2], [0.3, 0.4]], [[0.1, 0.2], [0.3, 0.4]]) == 0.0
    assert oc.chi([[0.1, 0.2, 0.3]], [[0.103, 0.203, 0.303]]) == pytest.approx(0.003, rel=1e-9)
    assert oc.chi([[1.0, 2.0]], [[1.0, 4.0]]) == pytest.approx(math.sqrt(2.0), rel=1e-15)


def test_oracle_h_bar_by_hand(oc):
    assert oc.h_bar([0.5, 0.1, 0.3], [8.9, 9.0, 12.0]) == pytest.approx(0.2, rel=1e-15)


def _quad(x):
    return (x[0] - 0.0061) ** 2 / 0.0025 ** 2 + (x[1] - 68.3) ** 2 / 4.0 ** 2 + 0.3 * (x[0] - 0.0061) * (x[1] - 68.3) / 0.01


LO, HI = [0.0025, 55.0], [0.0185, 80.0]


def test_oracle_pattern_search_quadratic(oc):
    x, fx, path, n = oc.hooke_jeeves(_quad, [0.0105, 67.5], [0.004, 6.25], LO, HI, tol=1e-5)
    assert abs(x[0] - 0.0061) < 2e-5 * 0.016 * 10 and abs(x[1] - 68.3) < 2e-5 * 25 * 10
    assert fx < 1e-6 and len(path) > 2


def test_oracle_pattern_search_boundary(oc):
    f = lambda x: (x[0] - 0.03) ** 2 * 1e4 + (x[1] - 60.0) ** 2      # alpha_s minimum outside the box
    x, fx, path, n = oc.hooke_jeeves(f, [0.0105, 67.5], [0.004, 6.25], LO, HI, tol=1e-6)
    assert x[0] == pytest.approx(0.0185, abs=1e-9) and x[1] == pytest.approx(60.0, abs=1e-3)


def test_oracle_pattern_search_path_by_hand(oc):
    """f = (x - 0.9)^2 + (y - 0.5)^2 on the unit box from (0.5, 0.5), step 0.1: the first
    exploration accepts x = 0.6; the pattern point 0.7 explores to 0.8 (accepted), the
    next pattern point 1.0 explores to 0.9 (accepted, f = 0), the one after fails; the
    halved steps find nothing lower."""
    f = lambda x: (x[0] - 0.9) ** 2 + (x[1] - 0.5) ** 2
    x, fx, path, n = oc.hooke_jeeves(f, [0.5, 0.5], [0.1, 0.1], [0.0, 0.0], [1.0, 1.0], tol=0.01)
    assert len(path) == 4
    assert np.allclose(path, [[0.5, 0.5], [0.6, 0.5], [0.8, 0.5], [0.9, 0.5]], rtol=0, atol=1e-12)
    assert fx < 1e-30


MUTANTS = {
    "no_minus_step": ("            t = list(x)\n            t[i] = x[i] - s[i]\n            ft = F(t)\n            if ft < fx:\n                x, fx = t, ft\n",
                      ""),
    "pattern_without_difference": ("p = [b[i] + (b[i] - prev[i]) for i in range(d)]", "p = [b[i] for i in range(d)]"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_oracle_pattern_search_mutants_fail_a_pin(oc, name):
    src = open(os.path.join(ROOT, "oracle", "calib.py")).read()
    old, new = MUTANTS[name]
    assert old in src
    mod = types.ModuleType("calib_mutant")
    exec(compile(src.replace(old, new), "calib_mutant", "exec"), mod.__dict__)
    failed = 0
    for pin in (test_oracle_pattern_search_quadratic, test_oracle_pattern_search_boundary,
                test_oracle_pattern_search_path_by_hand):
        try:
            pin(mod)
        except AssertionError:
            failed += 1
    assert failed >= 1, f"mutant {name} passes every pattern-search pin"


# ----------------------------------------------------------------------------- library against oracle

def test_sensitivity_chi_h_bar_match_oracle(oc):
    rng = np.random.default_rng(5)
    a_s, a_p, ds, dp = _grid()
    H = 0.1 + 0.01 * rng.random((len(a_s), len(a_p)))
    s0, p0 = oc.sensitivity(H.tolist(), ds, dp)
    s1, p1 = C.sensitivity(H, ds, dp)
    assert s1 == pytest.approx(s0, rel=1e-12) and p1 == pytest.approx(p0, rel=1e-12)
    he, hs = rng.random((6, 17)), rng.random((6, 17))
    assert C.chi(he, hs) == pytest.approx(oc.chi(he.tolist(), hs.tolist()), rel=1e-13)
    sc = inputs.flume(0.015, 1)
    h = rng.random((sc.rows, sc.cols)).astype(np.float32)
    x, _ = inputs.cell_centres(sc.rows, sc.cols, sc.l)
    assert C.h_bar(h, sc) == pytest.approx(oc.h_bar(h.ravel().tolist(), x.ravel().tolist()), rel=1e-13)


@pytest.mark.parametrize("case", ["quadratic", "boundary", "valley"])
def test_batched_pattern_search_takes_the_oracle_path(oc, case):
    f = {"quadratic": _quad,
         "boundary": lambda x: (x[0] - 0.03) ** 2 * 1e4 + (x[1] - 60.0) ** 2,
         "valley": lambda x: (x[1] / 25.0 - 2.2 - 400.0 * x[0] ** 2) ** 2 + 0.1 * (x[0] - 0.01) ** 2 / 0.0025 ** 2}[case]
    x0, step = [0.0105, 67.5], [0.004, 6.25]
    x_o, f_o, path_o, _ = oc.hooke_jeeves(f, x0, step, LO, HI, tol=1e-4)
    batches = []

    def f_batch(points):
        batches.append(len(points))
        return [f(p) for p in points]

    r = C.hooke_jeeves(f_batch, x0, step, LO, HI, tol=1e-4)
    assert len(r.path) == len(path_o)
    for a, b in zip(r.path, path_o):
        assert np.allclose(a, b, rtol=0, atol=1e-12)
    assert r.f == f_o and np.allclose(r.x, x_o, rtol=0, atol=1e-12)
    assert r.batches == len(batches) and max(batches) <= 9


# ----------------------------------------------------------------------------- flume inputs

def _west_width_brute(rows, l):
    """Sum of l (n_W . n) over the boundary edges whose missing neighbour lies west (the
    neighbour's row inside the raster, its column outside)."""
    n1 = [1.0, 0.5, -0.5, -1.0, -0.5, 0.5]
    total = 0.0
    for r in range(rows):
        odd = r & 1
        for d, (dr, dc) in enumerate([(0, 1), (1, odd), (1, odd - 1), (0, -1), (-1, odd - 1), (-1, odd)]):
            rr, cc = r + dr, 0 + dc
            if 0 <= rr < rows and cc < 0:
                total += l * (-1.0) * n1[d]
    return total


@pytest.mark.parametrize("rows", [2, 3, 6, 7, 10])
def test_flume_inflow_width(rows):
    assert inputs.west_width(rows, 0.1) == pytest.approx(_west_width_brute(rows, 0.1), rel=1e-14)


def test_flume_inflow_booked_by_the_oracle(orc):
    sc = inputs.flume(0.015, 1, t_end=5.0)
    sc.bc = (inputs.FLUX, inputs.WALL, inputs.WALL, inputs.WALL)
    p = orc.from_scenario(sc)
    r = p.run(p.mass(sc.h0), sc.v1_0.ravel().astype(float), sc.v2_0.ravel().astype(float), 0.0, 5.0)
    assert -r["ledger"].outflow == pytest.approx(0.015 * 5.0, rel=1e-9)


def test_flume_settles_with_viscosity(orc):
    """h changes by less than 1e-5 m over the last 100 s of a 600 s run (q = 21 l/s, the
    largest discharge of the vegetated-downstream layout)."""
    sc = inputs.flume(0.021, 1)
    sc.viscosity = True
    p = orc.from_scenario(sc)
    m, a, b = p.mass(sc.h0), sc.v1_0.ravel().astype(float), sc.v2_0.ravel().astype(float)
    r1 = p.run(m, a, b, 0.0, 500.0)
    r2 = p.run(r1["m"], r1["v1"], r1["v2"], r1["t"], 600.0)
    th = sc.theta.ravel().astype(float)
    assert np.max(np.abs(r2["m"] / th - r1["m"] / th)) < 1e-5


def test_flume_environment_overrides():
    sc = inputs.flume(0.015, 1, theta_v=0.98, slope=3.0e-3)
    x, _ = inputs.cell_centres(sc.rows, sc.cols, sc.l)
    assert np.all(sc.theta[x >= 9.0] == np.float32(0.98)) and np.all(sc.theta[x < 9.0] == 1.0)
    assert np.allclose(sc.z, (3.0e-3 * (18.0 - x)).astype(np.float32))
    d = inputs.flume(0.015, 2)
    assert np.all(d.theta[x < 9.0] == np.float32(inputs.FLUME["theta_v"])) and np.all(d.theta[x >= 9.0] == 1.0)
