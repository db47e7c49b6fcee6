"""The OpenMP build of the oracle gives bit for bit the single-threaded result: every
cell's update reads only the state at t^n, and the step's outflow and clamp sums are
formed after the cell loop in the single-threaded order.  Three rasters cover every
boundary type (wall, free discharge on an interval, given mass flux, Dirichlet), rain,
per-cell porosity, the artificial viscosity and the linear resistance with a dry
threshold; the runs take their own CFL steps and record a hydrograph."""
import numpy as np
import pytest

import oracle
from paper_2406_14933_gb300 import inputs

WALL, FREE, FLUX, DIR = 0, 1, 2, 3


def _cases():
    a = inputs.tiny(37, 53, 101, bc=(FREE, FREE, WALL, FREE), rain_mm_h=80.0)
    a.free_range = ((5, 30), (0, 0), (0, 0), (10, 40))
    b = inputs.tiny(40, 61, 202, bc=(FLUX, DIR, FREE, WALL), rain_mm_h=20.0, smooth=True)
    b.bc_q = (0.02, 0.0, 0.0, 0.0)
    b.bc_h = (0.0, 0.03, 0.0, 0.0)
    b.bc_u = (0.0, 0.1, 0.0, 0.0)
    b.viscosity = True
    c = inputs.tiny(33, 47, 303, bc=(DIR, WALL, FLUX, FREE))
    c.bc_h = (0.04, 0.0, 0.0, 0.0)
    c.bc_u = (0.2, 0.0, 0.0, 0.0)
    c.bc_q = (0.0, 0.0, 0.01, 0.0)
    c.tau = 0.3
    c.h_dry = 1e-3
    return [a, b, c]


@pytest.mark.parametrize("k", [0, 1, 2])
def test_openmp_build_is_bitwise_single_thread(k):
    sc = _cases()[k]
    out = []
    for threads in (1, 4):
        p = oracle.from_scenario(sc, threads=threads)
        res = p.run(p.mass(sc.h0), sc.v1_0, sc.v2_0, 0.0, 30.0, sample_dt=2.0, sample_cap=64)
        led = res["ledger"]
        out.append((res, (led.rain_in, led.outflow, led.clamped, led.steps),
                    p.cmax(res["m"], res["v1"], res["v2"]), p.cfl_dt(res["m"], res["v1"], res["v2"])))
    (r1, l1, c1, d1), (r4, l4, c4, d4) = out
    assert r1["steps"] == r4["steps"] > 10 and r1["t"] == r4["t"]
    for key in ("m", "v1", "v2", "samples"):
        assert np.array_equal(r1[key], r4[key]), key
    assert l1 == l4 and c1 == c4 and d1 == d4
    assert l1[1] != 0.0                       # water crossed the open sides


def test_thread_count_reported():
    p = oracle.from_scenario(_cases()[0], threads=3)
    p.cmax(p.mass(p.theta * 0.0 + 0.01), np.zeros(p.n), np.zeros(p.n))
    assert oracle.oracle._load(3).orc_threads(0) == 3
