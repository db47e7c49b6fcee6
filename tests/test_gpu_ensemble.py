"""The batched ensemble (one persistent launch, per-scenario clocks) against single
rasters and the oracle."""
import numpy as np
import pytest

from paper_2406_14933_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [40, 57, 90, 131, 200, 33]


def _scenarios(t_end=120.0, sample_dt=10.0):
    out = []
    for i, n in enumerate(SIZES):
        sc = inputs.ensemble_member(i, n_override=n, t_end=t_end)
        sc.sample_dt = sample_dt
        out.append(sc)
    return out


def _rel_l2(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def test_ensemble_matches_single_rasters_bitwise(asx, monkeypatch):
    """Each scenario of the ensemble reaches the same state, bit for bit, as the same
    raster run alone with the gather kernel (same per-cell code, same time steps)."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    from paper_2406_14933_gb300.raster import Raster
    monkeypatch.setenv("ASX_STEP_KERNEL", "gather")
    scs = _scenarios()
    E = Ensemble(scs)
    E.run()
    for i, sc in enumerate(scs):
        R = Raster(sc)
        t = R.run_until(sc.t_end)
        te, ke = E.clock(i)
        assert te == t == sc.t_end
        assert ke == R.clock()[2]
        for a, b in zip(E.state(i), R.state()):
            assert np.array_equal(a, b)
        le, lr = E.ledger(i), R.ledger()
        assert le.rain_in == pytest.approx(lr.rain_in, rel=1e-12)
        assert le.outflow == pytest.approx(lr.outflow, rel=1e-12, abs=1e-12)
        assert le.storage == pytest.approx(lr.storage, rel=1e-12)
        assert le.defect_rel <= 1e-10
        qe, qr = E.hydrograph(i), R.hydrograph()
        assert len(qe) == len(qr) == 12
        assert np.allclose(qe, qr, rtol=1e-10, atol=1e-14)
        R.close()
    E.close()


@pytest.mark.parametrize("tuning", [(1, 128, 1), (2, 256, 4), (8, 512, 2)])
def test_ensemble_launch_shapes_agree(asx, tuning):
    """Cluster size, threads and cells per thread change who computes a cell, not what:
    the states are identical for every launch shape."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    scs = _scenarios(t_end=60.0)
    E = Ensemble(scs)
    E.run((4, 256, 2))
    ref = [E.state(i) for i in range(len(scs))]
    E.run(tuning)
    for i in range(len(scs)):
        for a, b in zip(E.state(i), ref[i]):
            assert np.array_equal(a, b)
    E.close()


def test_ensemble_autotune_and_oracle(asx, orc):
    """The autotuner returns a valid launch shape; two scenarios match the FP64 oracle
    (own time steps on both sides) to the stated tolerance and close their budgets."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    scs = _scenarios(t_end=90.0)
    E = Ensemble(scs)
    t = E.autotune(max_steps=20)
    assert t.cluster in (1, 2, 4, 8) and t.threads in (128, 256, 512) and t.cells_per_thread in (1, 2, 4)
    assert t.tile_rows in (0, 1, 8, 16, 32) and t.split >= 0
    E.run()
    for i in (1, 4):
        sc = scs[i]
        p = orc.from_scenario(sc)
        # the same sample times cut the steps on both sides
        res = p.run(p.mass(sc.h0), sc.v1_0, sc.v2_0, 0.0, sc.t_end, sample_dt=sc.sample_dt,
                    sample_cap=100)
        mh, ml, v1, v2 = E.state(i)
        mg = mh.astype(np.float64) + ml
        assert _rel_l2(p.depth(mg.ravel()), p.depth(res["m"])) <= 1e-4
        qo = np.concatenate([res["m"] * res["v1"], res["m"] * res["v2"]])
        qg = np.concatenate([mg.ravel() * v1.ravel(), mg.ravel() * v2.ravel()])
        assert _rel_l2(qg, qo) <= 1e-4
        assert E.ledger(i).defect_rel <= 1e-10
        qh = np.diff(np.concatenate([[0.0], res["samples"]])) / sc.sample_dt
        assert _rel_l2(E.hydrograph(i), qh) <= 1e-4
    E.close()


def test_ensemble_tuning_after_a_complete_run(asx):
    """After a run that takes every scenario to its end, the autotuner cuts the scenarios in
    proportion to their measured step counts and the queue takes them by measured work;
    neither changes what a run computes: the states, clocks and ledgers of the next run are
    those of the first, bit for bit."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    scs = _scenarios(t_end=90.0)
    E = Ensemble(scs)
    E.run((2, 256, 2))
    ref = [(E.state(i), E.clock(i), E.ledger(i).outflow) for i in range(len(scs))]
    assert all(c[0] == sc.t_end for (_, c, _), sc in zip(ref, scs))
    t = E.autotune(max_steps=5)
    assert t.cluster in (1, 2, 4, 8) and t.threads in (128, 256, 512) and t.cells_per_thread in (1, 2, 4)
    assert t.tile_rows in (0, 1, 8, 16, 32) and t.split >= 0
    E.run((2, 256, 2))
    for i in range(len(scs)):
        st, clk, out = ref[i]
        for a, b in zip(E.state(i), st):
            assert np.array_equal(a, b)
        assert E.clock(i) == clk
        assert E.ledger(i).outflow == out
    E.run()
    for i in range(len(scs)):
        assert E.clock(i) == ref[i][1]
    E.close()


# sides wide enough for strip tiles (an overlapping last strip at 200, 173 and 300; the
# narrowest case with tensor maps, 144; rows left to the frame), and one all-frame raster
STRIP_SIZES = [200, 300, 173, 144, 40, 261]


def _strip_scenarios(t_end=60.0, sample_dt=10.0):
    out = []
    for i, n in enumerate(STRIP_SIZES):
        sc = inputs.ensemble_member(20 + i, n_override=n, t_end=t_end)
        sc.sample_dt = sample_dt
        out.append(sc)
    return out


@pytest.mark.parametrize("tile_rows", [8, 16, 32])
def test_strip_ensemble_matches_single_rasters_bitwise(asx, monkeypatch, tile_rows):
    """The strip ensemble kernel gives every cell the code the single raster's strip kernel
    gives it in the same layout (the tile code inside, the gather code on the frame): each
    scenario reaches the state of the same raster run alone with the strip kernel at the
    same tile height, bit for bit, with the same time steps and hydrograph."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    from paper_2406_14933_gb300.raster import Raster
    monkeypatch.delenv("ASX_STEP_KERNEL", raising=False)
    monkeypatch.setenv("ASX_TILE_ROWS", str(tile_rows))
    scs = _strip_scenarios()
    E = Ensemble(scs)
    E.run((2, 256, 1, tile_rows))
    for i, sc in enumerate(scs):
        R = Raster(sc)
        t = R.run_until(sc.t_end)
        te, ke = E.clock(i)
        assert te == t == sc.t_end
        assert ke == R.clock()[2]
        for a, b in zip(E.state(i), R.state()):
            assert np.array_equal(a, b)
        le, lr = E.ledger(i), R.ledger()
        # the boundary sums are added in another order
        assert le.rain_in == pytest.approx(lr.rain_in, rel=1e-12)
        assert le.outflow == pytest.approx(lr.outflow, rel=1e-12, abs=1e-12)
        assert le.storage == pytest.approx(lr.storage, rel=1e-12)
        assert le.defect_rel <= 1e-10
        qe, qr = E.hydrograph(i), R.hydrograph()
        assert len(qe) == len(qr) == 6
        assert np.allclose(qe, qr, rtol=1e-10, atol=1e-14)
        R.close()
    E.close()


@pytest.mark.parametrize("tuning", [(1, 128, 1, 16), (4, 128, 1, 16), (8, 256, 1, 16), (4, 256, 1, 16, 2),
                                    (8, 128, 1, 16, 5), (2, 512, 1, 16)])
def test_strip_ensemble_launch_shapes_agree(asx, tuning):
    """Cluster size, tile workers per CTA and the split (the largest scenarios on whole
    clusters, the rest on single CTAs) change which warp computes a tile, not what: the
    states are identical for every strip launch shape of one tile height."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    scs = _strip_scenarios(t_end=40.0)
    E = Ensemble(scs)
    E.run((2, 256, 1, 16))
    ref = [E.state(i) for i in range(len(scs))]
    E.run(tuning)
    for i in range(len(scs)):
        for a, b in zip(E.state(i), ref[i]):
            assert np.array_equal(a, b)
    E.close()


@pytest.mark.parametrize("tuning", [(4, 256, 1, 1), (4, 256, 1, 1, 2)])
def test_strip_ensemble_tile_height_per_scenario(asx, monkeypatch, tuning):
    """With the tile height chosen per scenario (tile_rows = 1; with and without a split),
    each scenario equals, bit for bit and step for step, the single raster run by the strip
    kernel at one of the heights 8, 16, 32."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    from paper_2406_14933_gb300.raster import Raster
    monkeypatch.delenv("ASX_STEP_KERNEL", raising=False)
    scs = _strip_scenarios(t_end=30.0)
    E = Ensemble(scs)
    E.run(tuning)
    got = [(E.state(i), E.clock(i)) for i in range(len(scs))]
    E.close()
    for i, sc in enumerate(scs):
        match = False
        for h in (8, 16, 32):
            monkeypatch.setenv("ASX_TILE_ROWS", str(h))
            R = Raster(sc)
            R.run_until(sc.t_end)
            same = R.clock()[2] == got[i][1][1] and all(np.array_equal(a, b) for a, b in zip(R.state(), got[i][0]))
            R.close()
            if same:
                match = True
                break
        assert match, f"scenario {i} matches no single-raster tile height"


@pytest.mark.parametrize("tuning", [(2, 256, 1, 16), (4, 128, 1, 8, 1)])
def test_strip_ensemble_optional_terms_and_inflow(asx, monkeypatch, tuning):
    """The strip ensemble kernel with the optional terms compiled in (artificial viscosity,
    linear resistance, dry threshold) and a given-flux inflow side (frame code): each
    scenario equals the single raster run by the strip kernel at the same tile height, bit
    for bit, and its ledger books the inflow."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    from paper_2406_14933_gb300.raster import Raster
    monkeypatch.delenv("ASX_STEP_KERNEL", raising=False)
    monkeypatch.setenv("ASX_TILE_ROWS", str(tuning[3]))
    scs = []
    for i, n in enumerate((200, 150, 261)):
        sc = inputs.ensemble_member(40 + i, n_override=n, t_end=40.0)
        sc.sample_dt = 10.0
        sc.viscosity = True
        sc.tau = 0.02
        sc.h_dry = 1.0e-4
        scs.append(sc)
    scs[0].bc = (inputs.FLUX, inputs.FREE, inputs.WALL, inputs.WALL)
    scs[0].bc_q = (0.01, 0.0, 0.0, 0.0)
    E = Ensemble(scs)
    E.run(tuning)
    for i, sc in enumerate(scs):
        R = Raster(sc)
        R.run_until(sc.t_end)
        assert E.clock(i)[1] == R.clock()[2]
        for a, b in zip(E.state(i), R.state()):
            assert np.array_equal(a, b)
        assert E.ledger(i).defect_rel <= 1e-10
        R.close()
    assert E.ledger(0).outflow < 0.0           # the inflow side feeds more than leaves
    E.close()


def test_strip_ensemble_against_oracle(asx, orc):
    """Two strip-ensemble scenarios (tiles and frame) against the FP64 oracle on their own
    time steps, to the stated tolerance, with closed budgets."""
    from paper_2406_14933_gb300.ensemble import Ensemble
    scs = _strip_scenarios(t_end=90.0)
    E = Ensemble(scs)
    E.run((4, 256, 1, 8))
    for i in (0, 2):
        sc = scs[i]
        p = orc.from_scenario(sc)
        res = p.run(p.mass(sc.h0), sc.v1_0, sc.v2_0, 0.0, sc.t_end, sample_dt=sc.sample_dt, sample_cap=100)
        mh, ml, v1, v2 = E.state(i)
        mg = mh.astype(np.float64) + ml
        assert _rel_l2(p.depth(mg.ravel()), p.depth(res["m"])) <= 1e-4
        qo = np.concatenate([res["m"] * res["v1"], res["m"] * res["v2"]])
        qg = np.concatenate([mg.ravel() * v1.ravel(), mg.ravel() * v2.ravel()])
        assert _rel_l2(qg, qo) <= 1e-4
        assert E.ledger(i).defect_rel <= 1e-10
        qh = np.diff(np.concatenate([[0.0], res["samples"]])) / sc.sample_dt
        assert _rel_l2(E.hydrograph(i), qh) <= 1e-4
    E.close()


@pytest.mark.parametrize("tuning", [(2, 1024, 1, 16), (2, 256, 2, 16), (2, 256, 1, 12), (3, 256, 1, 16),
                                    (2, 1024, 1, 1), (2, 256, 1, 2), (2, 256, 1, 16, -1), (1, 256, 1, 16, 2),
                                    (2, 256, 2, 0, 2)])
def test_ensemble_rejects_bad_strip_shapes(asx, tuning):
    from paper_2406_14933_gb300.asx import AsxError, ASX_EINVAL
    from paper_2406_14933_gb300.ensemble import Ensemble
    E = Ensemble(_strip_scenarios(t_end=10.0)[:2])
    with pytest.raises(AsxError) as ei:
        E.run(tuning)
    assert ei.value.status == ASX_EINVAL
    E.close()


def test_ensemble_inflow_boundary_matches_single_raster(asx, monkeypatch):
    """A scenario fed through a given-mass-flux side runs in the ensemble exactly as a
    single raster with the gather kernel (bit for bit), the inflow booked alike."""
    import numpy as np
    from paper_2406_14933_gb300 import inputs
    from paper_2406_14933_gb300.ensemble import Ensemble
    from paper_2406_14933_gb300.raster import Raster
    monkeypatch.setenv("ASX_STEP_KERNEL", "gather")
    sc = inputs.ensemble_member(5, n_override=96, t_end=60.0)
    sc.bc = (inputs.FLUX, inputs.FREE, inputs.WALL, inputs.WALL)
    sc.bc_q = (0.01, 0.0, 0.0, 0.0)
    sc2 = inputs.ensemble_member(6, n_override=64, t_end=40.0)
    E = Ensemble([sc, sc2])
    E.run()
    R = Raster(sc)
    R.run_until(sc.t_end)
    for a, b in zip(E.state(0), R.state()):
        assert np.array_equal(a, b)
    le, lr = E.ledger(0), R.ledger()
    assert le.outflow == lr.outflow and le.outflow < 0.0
    E.close()
    R.close()
