"""The flume study of Sec. 4.3 on the GPU: the ensemble with the optional terms against
single rasters (bit for bit) and the oracle, the sensitivities of a small grid against
the oracle's, the full 21 x 26 grid, and the recovery of known friction coefficients by
the pattern search from solver-made gauges.

Tolerances: depths after 300 s of flume flow, relative L2 <= 1e-4 (the stated one).  The
sensitivities divide differences of h_bar between neighbouring grid points (a few mm
over the grid, against float32 errors of ~1e-6 m in h_bar) by the grid step: a relative
error of 1e-3 leaves a margin of ~10.
"""
import numpy as np
import pytest

from paper_2406_14933_gb300 import calibration as C
from paper_2406_14933_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _oracle_depth(orc, sc):
    p = orc.from_scenario(sc)
    r = p.run(p.mass(sc.h0), sc.v1_0.ravel().astype(float), sc.v2_0.ravel().astype(float), 0.0, sc.t_end)
    return (r["m"] / sc.theta.ravel().astype(float)).reshape(sc.rows, sc.cols), r


def test_ensemble_optional_terms_match_single_raster(asx, monkeypatch):
    """Flume scenarios with the artificial viscosity (and, in a second one, the linear
    resistance and dry threshold) reach the same state in the ensemble, bit for bit, as a
    single raster with the gather kernel, the budget booked alike."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    from paper_2406_14933_gb300.raster import Raster
    monkeypatch.setenv("ASX_STEP_KERNEL", "gather")
    a = inputs.flume(0.015, 1, t_end=20.0)
    a.viscosity = True
    b = inputs.flume(0.05, 2, alpha_s=0.012, alpha_p=60.0, l=0.15, t_end=15.0)
    b.viscosity, b.tau, b.h_dry = True, 0.05, 1e-3
    plain = inputs.ensemble_member(3, n_override=48, t_end=30.0)
    E = Ensemble([a, plain, b])
    E.run()
    for i, sc in [(0, a), (2, b)]:
        R = Raster(sc)
        R.run_until(sc.t_end)
        for x, y in zip(E.state(i), R.state()):
            assert np.array_equal(x, y)
        le, lr = E.ledger(i), R.ledger()
        assert le.outflow == lr.outflow
        R.close()
    E.close()


@pytest.mark.parametrize("exp", [(1, 0.015, 0.00709, 73.39), (2, 0.05, 0.015, 58.0)])
def test_flume_depths_against_oracle(asx, orc, exp):
    layout, q, a_s, a_p = exp
    study = C.FlumeStudy(l=0.2, t_end=300.0)
    sc = study.scenario(a_s, a_p, layout, q)
    h_gpu = C.steady_depths(study, [sc])[0]
    h_orc, _ = _oracle_depth(orc, sc)
    e = _rel_l2(h_gpu, h_orc)
    print(f"[flume] layout {layout} q {q}: depth rel L2 {e:.2e}")
    assert e <= 1e-4


def test_sensitivity_subgrid_against_oracle(asx, orc):
    """delta_s, delta_p of a 3 x 3 grid over the search box (layout 1, 15 l/s), from the
    ensemble and from the oracle's h_bar with the oracle's double sums."""
    import oracle.calib as oc
    study = C.FlumeStudy(l=0.2, t_end=300.0)
    r = C.sensitivity_grid(study, 1, 0.015, ns=3, np_=3)
    Ho = []
    for s in r["alpha_s"]:
        row = []
        for p in r["alpha_p"]:
            sc = study.scenario(s, p, 1, 0.015)
            h, _ = _oracle_depth(orc, sc)
            x, _ = inputs.cell_centres(sc.rows, sc.cols, sc.l)
            row.append(oc.h_bar(h.ravel().tolist(), x.ravel().tolist()))
        Ho.append(row)
    ds_o, dp_o = oc.sensitivity(Ho, r["alpha_s"][1] - r["alpha_s"][0], r["alpha_p"][1] - r["alpha_p"][0])
    print(f"[sensitivity] GPU {r['delta_s']:.6g} {r['delta_p']:.6g}  oracle {ds_o:.6g} {dp_o:.6g}")
    assert np.allclose(r["h_bar"], Ho, rtol=1e-5, atol=0)
    assert r["delta_s"] == pytest.approx(ds_o, rel=1e-3) and r["delta_p"] == pytest.approx(dp_o, rel=1e-3)


def test_sensitivity_full_grid(asx):
    """The 21 x 26 grid of Sec. 4.3 on the default flume (546 scenarios in one ensemble):
    more friction of either kind raises the mean depth of the vegetated reach, and the
    grid is steady (h_bar changes by less than 1e-5 m when the runs go on 60 s longer, on
    the grid's corners)."""
    study = C.FlumeStudy()
    r = C.sensitivity_grid(study, 1, 0.015)
    assert r["h_bar"].shape == (21, 26)
    assert r["delta_s"] > 0.0 and r["delta_p"] > 0.0
    longer = C.FlumeStudy(t_end=study.t_end + 60.0)
    corners = [(r["alpha_s"][i], r["alpha_p"][j]) for i in (0, -1) for j in (0, -1)]
    scs = [longer.scenario(s, p, 1, 0.015) for s, p in corners]
    hs = C.steady_depths(longer, scs)
    for (i, j), h, sc in zip([(0, 0), (0, -1), (-1, 0), (-1, -1)], hs, scs):
        assert abs(C.h_bar(h, sc) - r["h_bar"][i, j]) < 1e-5
    print(f"[sensitivity] 21x26 grid: delta_s {r['delta_s']:.4g} m, delta_p {r['delta_p']:.4g} m^2, "
          f"{study.runs} runs in {study.seconds:.2f} s")


def test_calibration_recovers_known_coefficients(asx):
    """Gauges made by the solver at (0.00709, 73.39), all six experiments: the pattern
    search from the centre of the box ends within 2 % of the box's span of the known pair,
    with a misfit below 0.1 mm."""
    study = C.FlumeStudy(l=0.2, t_end=400.0)
    truth = (0.00709, 73.39)
    h_exp = C.synthetic_gauges(study, *truth)
    r = C.calibrate(study, h_exp, tol=2e-3)
    print(f"[calibration] found {r.x} chi {r.f:.3g} m, {r.evals} points in {r.batches} batches, "
          f"{study.runs} runs, {study.seconds:.2f} s")
    assert abs(r.x[0] - truth[0]) <= 0.02 * (C.LAMBDA[0][1] - C.LAMBDA[0][0])
    assert abs(r.x[1] - truth[1]) <= 0.02 * (C.LAMBDA[1][1] - C.LAMBDA[1][0])
    assert r.f < 1e-4


def test_sensitivity_sweep_over_environments(asx):
    """delta_s, delta_p over environments p = (q, theta_v, m), every grid in one ensemble:
    without vegetation (theta_v = 1) the plant drag alpha_p (1 - theta) vanishes, every
    alpha_p gives the same run bit for bit and delta_p is exactly 0; with vegetation it is
    positive; and an environment's grid inside the sweep is, bit for bit, the grid run on
    its own."""
    study = C.FlumeStudy(l=0.2, t_end=300.0)
    envs = [dict(q=0.015), dict(q=0.015, theta_v=1.0), dict(q=0.007, slope=3.0e-3)]
    res = C.sensitivity_sweep(study, envs, ns=5, np_=5)
    assert res[1]["delta_p"] == 0.0
    assert res[0]["delta_p"] > 0.0 and res[2]["delta_p"] > 0.0
    alone = C.sensitivity_grid(C.FlumeStudy(l=0.2, t_end=300.0), 1, 0.015, ns=5, np_=5)
    assert np.array_equal(alone["h_bar"], res[0]["h_bar"])
    for r in res:
        print(f"[sweep] {r['env']}: delta_s {r['delta_s']:.4g} m, delta_p {r['delta_p']:.4g} m^2")


def test_chi_surfaces_of_the_four_cases(asx):
    """chi over the 21 x 26 grid for the experiment subsets of Sec. 4.3 (I: one experiment,
    II / III: the three of one vegetation layout, IV: all six), gauges made by the solver at
    (0.00709, 73.39): the grid minimum of case IV lies within one grid step of that pair.
    The size of each case's low-misfit region (chi below twice the grid's lowest value plus
    0.1 mm) is printed: the paper finds one experiment locates the minimum poorly and all
    six best."""
    study = C.FlumeStudy(l=0.2, t_end=400.0)
    truth = (0.00709, 73.39)
    h_exp = C.synthetic_gauges(study, *truth)
    r = C.chi_surfaces(study, h_exp)
    ds, dp = r["alpha_s"][1] - r["alpha_s"][0], r["alpha_p"][1] - r["alpha_p"][0]
    am = r["cases"]["IV"]["argmin"]
    assert abs(am[0] - truth[0]) <= ds * 1.0001 and abs(am[1] - truth[1]) <= dp * 1.0001
    for name, c in r["cases"].items():
        low = int((c["chi"] <= 2.0 * c["min"] + 1e-4).sum())
        print(f"[cases] {name}: grid minimum {c['min'] * 1e3:.3f} mm at {c['argmin']}, {low} of 546 points low")
