"""The FP64 mode (asx_raster_desc.precision = ASX_FP64) and the float64 bed.

In FP64 mode the state, bed and porosity are float64 and every operation rounds as
written (no fused multiply-adds), each operator summed over a cell's neighbours in the
oracle's direction order: the GPU run follows the FP64 oracle to rounding.  Over whole
runs with their own time steps on both sides the two are held to 1e-12 relative L2 in
depth and discharge (the FP32 mode's bound is 1e-4); the water budget closes to 1e-12.

The bed enters as float64 in both modes: the FP32 mode rounds it to the nearest float32
(round to nearest even), which a run with the same bed given already rounded reproduces
bit for bit, from host or device pointers alike.
"""
import numpy as np
import pytest

from paper_2406_14933_gb300 import inputs

pytestmark = pytest.mark.gpu

WALL, FREE, FLUX, DIR = 0, 1, 2, 3


def _rel_l2(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _compare(sc, R, res):
    h, v1, v2 = R.fields64()
    theta = np.asarray(sc.theta, np.float64).ravel()
    ho = res["m"] / theta
    eh = _rel_l2(h.ravel(), ho)
    qg = np.concatenate([(h.ravel() * theta) * v1.ravel(), (h.ravel() * theta) * v2.ravel()])
    qo = np.concatenate([res["m"] * res["v1"], res["m"] * res["v2"]])
    return eh, _rel_l2(qg, qo)


def test_fp64_hillslope_whole_run(asx, orc):
    """The 64 x 64 hillslope (5 % slope, porosity 0.9, 50 mm/h for 600 s, free east side),
    both sides from the dry start to t_end = 600 s with their own CFL steps."""
    from paper_2406_14933_gb300.raster import Raster
    sc = inputs.hillslope()
    R = Raster(sc, fp64=True)
    assert R.run_until(sc.t_end) == sc.t_end
    steps = R.clock()[2]
    led = R.ledger()
    p = orc.from_scenario(sc)
    res = p.run(p.mass(sc.h0), sc.v1_0, sc.v2_0, 0.0, sc.t_end)
    eh, eq = _compare(sc, R, res)
    print(f"[fp64] hillslope 64^2 to {sc.t_end:.0f} s: GPU {steps} steps, oracle {res['steps']}; "
          f"depth {eh:.2e} discharge {eq:.2e} defect {led.defect_rel:.1e}")
    assert steps == res["steps"]
    assert eh <= 1e-12 and eq <= 1e-12
    assert led.defect_rel <= 1e-12
    assert led.rain_in == pytest.approx(res["ledger"].rain_in, rel=1e-13)
    assert led.outflow == pytest.approx(res["ledger"].outflow, rel=1e-11)
    R.close()


@pytest.mark.parametrize("case", ["flux_dirichlet_viscosity", "classes_free_interval", "tau_dry"])
def test_fp64_every_term(asx, orc, case):
    from paper_2406_14933_gb300.raster import Raster
    if case == "flux_dirichlet_viscosity":
        sc = inputs.tiny(40, 61, 202, bc=(FLUX, DIR, FREE, WALL), rain_mm_h=20.0, smooth=True)
        sc.bc_q = (0.02, 0.0, 0.0, 0.0)
        sc.bc_h = (0.0, 0.03, 0.0, 0.0)
        sc.bc_u = (0.0, 0.1, 0.0, 0.0)
        sc.viscosity = True
    elif case == "classes_free_interval":
        sc = inputs.carved_catchment(rows=96, cols=80, l=20.0, block=16, min_acc=4)
        sc.h0 = np.full((sc.rows, sc.cols), 0.02, np.float32)
    else:
        sc = inputs.tiny(33, 47, 303, bc=(DIR, WALL, FLUX, FREE))
        sc.bc_h = (0.04, 0.0, 0.0, 0.0)
        sc.bc_u = (0.2, 0.0, 0.0, 0.0)
        sc.bc_q = (0.0, 0.0, 0.01, 0.0)
        sc.tau = 0.3
        sc.h_dry = 1e-3
    R = Raster(sc, fp64=True)
    t_end = 30.0
    R.run_until(t_end)
    steps = R.clock()[2]
    p = orc.from_scenario(sc)
    res = p.run(p.mass(sc.h0), sc.v1_0, sc.v2_0, 0.0, t_end, sample_dt=sc.sample_dt, sample_cap=64)
    eh, eq = _compare(sc, R, res)
    print(f"[fp64] {case}: GPU {steps} steps, oracle {res['steps']}; depth {eh:.2e} discharge {eq:.2e}")
    assert steps == res["steps"] > 20
    assert eh <= 1e-12 and eq <= 1e-12
    assert R.ledger().defect_rel <= 1e-12
    R.close()


def test_fp64_mode_readers(asx):
    """float32 fields are the rounded float64 ones; the compensated float32 state does not
    exist in FP64 mode; a precision other than the two modes is refused."""
    from paper_2406_14933_gb300 import asx as A
    from paper_2406_14933_gb300.raster import Raster
    sc = inputs.tiny(20, 30, 7, bc=(FREE, WALL, WALL, WALL), rain_mm_h=40.0)
    R = Raster(sc, fp64=True)
    R.step(10)
    h64, a64, b64 = R.fields64()
    h32, a32, b32 = R.fields()
    assert np.array_equal(h32, h64.astype(np.float32)) and np.array_equal(a32, a64.astype(np.float32))
    with pytest.raises(A.AsxError) as e:
        R.state()
    assert e.value.status == A.ASX_EINVAL
    R.close()
    d = A.asx_raster_desc()
    d.rows, d.cols, d.edge_m, d.precision = 8, 8, 1.0, 7
    with pytest.raises(A.AsxError) as e:
        A.asx_create_raster(d)
    assert e.value.status == A.ASX_EINVAL


@pytest.mark.parametrize("kind", ["host", "device"])
def test_fp32_mode_rounds_a_float64_bed(asx, kind):
    """A bed given in float64 with sub-float32 detail (a DEM at 1000 m with 1e-6 m
    features) runs exactly as the same bed rounded to float32 beforehand."""
    import torch
    from paper_2406_14933_gb300 import asx as A
    from paper_2406_14933_gb300.raster import Raster
    sc = inputs.tiny(40, 150, 9, bc=(FREE, FREE, WALL, WALL), rain_mm_h=30.0, smooth=True)
    rng = np.random.default_rng(3)
    z64 = 1000.0 + sc.z.astype(np.float64) + rng.uniform(-1e-6, 1e-6, sc.z.shape)
    assert not np.array_equal(z64, z64.astype(np.float32).astype(np.float64))
    out = []
    for z in (z64, z64.astype(np.float32).astype(np.float64)):
        R = Raster(sc)
        args = [z, sc.theta, None, sc.h0, sc.v1_0, sc.v2_0]
        if kind == "device":
            dev = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in args]
            A.asx_set_fields(R.handle, *dev, A.ASX_PTR_DEVICE)
            torch.cuda.synchronize()
        else:
            A.asx_set_fields(R.handle, *[None if a is None else np.ascontiguousarray(a) for a in args],
                             A.ASX_PTR_HOST)
        R.step(25)
        out.append(R.state())
        R.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
