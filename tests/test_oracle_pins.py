"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

None of these re-types the oracle's formulas: each checks a property that a dropped
term, a wrong sign, a wrong neighbour index or a transposed operand would break.
  * lake at rest stays at rest (well-balanced S term, Eq. fvm_2D_eq_frac.01, and the
    dry-island rule of Eq. fvm_2D_eq.05);
  * exact mass ledger: rain in = storage + outflow (flux antisymmetry; the identity
    rain - out = left printed for the Susita experiment, Table table_BasinSusita);
  * six-fold rotational and mirror symmetry of a radial dam break (geometry, normals,
    odd/even row neighbour offsets);
  * uniform sheet flow on a plane is an exact interior fixed point (S consistency with
    sum_j n_j n_j^T = 3 I and the friction balance K |v| v = theta h g s);
  * the closed-form friction solve satisfies alpha v + beta |v| v = gamma
    (Appendix A, Eq. miu-formula);
  * positivity for CFL <= 1 (Appendix A);
  * phi = area / perimeter of the regular hexagon (Eq. fvm_2D_eq_frac.13);
  * the rain volume of the Susita storm (Appendix C, Sec. 4.2.1) from the printed
    cell count and radius, independent of porosity;
  * a two-cell dam break worked by hand from Eqs. fvm_2D_eq.04-06 and fvm_2D_eq_frac.07.
"""
import math
import os

import numpy as np
import pytest

from paper_2406_14933_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _centres(rows, cols, l):
    x, y = inputs.cell_centres(rows, cols, l)
    return x.reshape(-1), y.reshape(-1)


def _smooth_bed(rows, cols, seed, relief):
    rng = np.random.default_rng(seed)
    x, y = _centres(rows, cols, 1.0)
    z = np.zeros(rows * cols)
    for _ in range(4):
        kx, ky, ph = rng.normal(0, 0.3), rng.normal(0, 0.3), rng.uniform(0, 2 * np.pi)
        z += np.cos(kx * x + ky * y + ph)
    z = relief * (z - z.min()) / (z.max() - z.min())
    return z


def test_lake_at_rest_wet(orc):
    """A flat free surface over a rough bed (everywhere wet, walls) stays at rest to
    rounding: after 200 steps |v| and |h - h0| are below 1e-12.  (With free-discharge
    sides the lake is only neutrally stable: outward rounding noise drains it, since the
    ghost copy gives no restoring pressure; the exact dyadic test below covers them.)"""
    bc = (0, 0, 0, 0)
    rows, cols = 24, 20
    z = _smooth_bed(rows, cols, 7, relief=1.0)
    rng = np.random.default_rng(3)
    theta = rng.uniform(0.5, 1.0, rows * cols)
    p = orc.Problem(rows, cols, 1.0, z, theta, alpha_s=rng.uniform(0, 0.02, rows * cols),
                    alpha_p=rng.uniform(0, 100, rows * cols), bc=bc)
    h0 = 1.3 - z
    assert h0.min() > 0.2
    res = p.run(p.mass(h0), 0.0, 0.0, 0.0, 1.0e9, max_steps=200)
    assert res["steps"] == 200
    assert np.abs(p.depth(res["m"]) - h0).max() <= 1e-12
    assert np.abs(res["v1"]).max() <= 1e-12 and np.abs(res["v2"]).max() <= 1e-12
    assert res["ledger"].outflow == 0.0


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1)])
def test_lake_at_rest_dry_islands(orc, bc):
    """A lake with dry islands stays exactly at rest: at a wet/dry edge v_n = 0, so the
    pressure term takes the mass of the higher side (Eq. fvm_2D_eq.05), which is the dry
    island's zero.  Bed, surface and porosity are dyadic so every difference is exact
    (with rounding noise in v the upwind branch of Eq. fvm_2D_eq.05 would be taken)."""
    rows, cols = 24, 20
    z = np.round(_smooth_bed(rows, cols, 7, relief=1.0) * 4096) / 4096
    rng = np.random.default_rng(3)
    theta = rng.choice([0.5, 0.625, 0.75, 0.875, 1.0], rows * cols)
    p = orc.Problem(rows, cols, 1.0, z, theta, alpha_s=rng.uniform(0, 0.02, rows * cols),
                    alpha_p=rng.uniform(0, 100, rows * cols), bc=bc)
    eta = 0.625
    h0 = np.maximum(eta - z, 0.0)
    assert (h0 == 0).sum() > 10 and (h0 > 0).sum() > 100
    res = p.run(p.mass(h0), 0.0, 0.0, 0.0, 1.0e9, max_steps=1000)
    assert res["steps"] == 1000
    assert np.abs(p.depth(res["m"]) - h0).max() == 0.0
    assert np.abs(res["v1"]).max() == 0.0 and np.abs(res["v2"]).max() == 0.0


def test_lake_at_rest_breaks_without_hat_rule(orc):
    """Sanity of the pin above: the same lake with a *sloping* surface does move."""
    rows, cols = 12, 12
    z = _smooth_bed(rows, cols, 7, relief=1.0)
    x, _ = _centres(rows, cols, 1.0)
    p = orc.Problem(rows, cols, 1.0, z, 1.0, 0.0, 0.0)
    h0 = np.maximum(1.5 + 0.01 * x - z, 0.0)
    res = p.run(p.mass(h0), 0.0, 0.0, 0.0, 1.0e9, max_steps=5)
    assert np.abs(res["v1"]).max() > 1e-4


@pytest.mark.parametrize("case", ["hillslope", "tiny_free"])
def test_mass_ledger_exact(orc, case):
    """Initial storage + rain in + clamped = storage + outflow, to rounding (FP64)."""
    if case == "hillslope":
        sc = inputs.hillslope()
        t_end = sc.t_end
    else:
        sc = inputs.tiny(17, 23, seed=5, bc=(1, 1, 1, 1), rain_mm_h=80.0)
        t_end = 200.0
    p = orc.from_scenario(sc)
    m0 = p.mass(sc.h0)
    s0 = p.storage(m0)
    res = p.run(m0, sc.v1_0, sc.v2_0, 0.0, t_end)
    L = res["ledger"]
    s1 = p.storage(res["m"])
    assert L.outflow > 0
    scale = max(L.rain_in, s0)
    defect = abs(s0 + L.rain_in + L.clamped - L.outflow - s1) / scale
    assert defect <= 1e-13, defect
    if case == "hillslope":
        # constant 50 mm/h over 64 x 64 cells of 1 m edge for 600 s
        area = 64 * 64 * 1.5 * math.sqrt(3.0)
        assert L.rain_in == pytest.approx(area * 50e-3 / 3600 * 600, rel=1e-12)


def _rotation_maps(rows, cols, l, centre):
    """Index maps of the 60-degree rotation and the x-mirror about a cell centre,
    found from centre coordinates (cells whose image leaves the raster map to -1)."""
    x, y = _centres(rows, cols, l)
    x0, y0 = x[centre], y[centre]
    key = {(round((xi - x0) / l, 6), round((yi - y0) / l, 6)): i
           for i, (xi, yi) in enumerate(zip(x, y))}
    c60, s60 = 0.5, math.sqrt(3.0) / 2
    rot = np.full(rows * cols, -1)
    mir = np.full(rows * cols, -1)
    for i in range(rows * cols):
        dx, dy = x[i] - x0, y[i] - y0
        rx, ry = c60 * dx - s60 * dy, s60 * dx + c60 * dy
        rot[i] = key.get((round(rx / l, 6), round(ry / l, 6)), -1)
        mir[i] = key.get((round(-dx / l, 6), round(dy / l, 6)), -1)
    return rot, mir


def test_sixfold_and_mirror_symmetry(orc):
    """A radially symmetric dam break centred on a cell stays six-fold and mirror
    symmetric (flat bed, uniform porosity and coefficients)."""
    rows, cols, l = 41, 41, 1.0
    centre = 20 * cols + 20
    x, y = _centres(rows, cols, l)
    d2 = (x - x[centre]) ** 2 + (y - y[centre]) ** 2
    h0 = 0.2 + 0.8 * np.exp(-d2 / 12.0)
    p = orc.Problem(rows, cols, l, 0.0, 0.85, alpha_s=0.01, alpha_p=30.0)
    res = p.run(p.mass(h0), 0.0, 0.0, 0.0, 1.0e9, max_steps=12)
    m, v1, v2 = res["m"], res["v1"], res["v2"]
    assert np.abs(v1).max() > 1e-2
    rot, mir = _rotation_maps(rows, cols, l, centre)
    near = np.sqrt(d2) <= 12.0 * l
    c60, s60 = 0.5, math.sqrt(3.0) / 2
    checked = 0
    for i in np.nonzero(near)[0]:
        j = rot[i]
        assert j >= 0
        assert abs(m[j] - m[i]) <= 1e-12
        assert abs(v1[j] - (c60 * v1[i] - s60 * v2[i])) <= 1e-12
        assert abs(v2[j] - (s60 * v1[i] + c60 * v2[i])) <= 1e-12
        k = mir[i]
        assert k >= 0
        assert abs(m[k] - m[i]) <= 1e-12
        assert abs(v1[k] + v1[i]) <= 1e-12 and abs(v2[k] - v2[i]) <= 1e-12
        checked += 1
    assert checked > 150


@pytest.mark.parametrize("theta,angle_deg", [(1.0, 0.0), (0.8, 17.0), (0.93, 200.0)])
def test_uniform_sheet_flow_fixed_point(orc, theta, angle_deg):
    """Uniform flow down a plane with K(h, theta)|v|^2 = theta h g s is an exact interior
    fixed point: cells further than k cells from the boundary do not change in k steps."""
    rows, cols, l, g, s = 30, 30, 2.0, 9.81, 0.04
    a_s, a_p = 0.00709, 73.39
    phi = math.radians(angle_deg)
    x, y = _centres(rows, cols, l)
    z = -s * (x * math.cos(phi) + y * math.sin(phi))
    h = 0.02
    K = a_p * h * (1.0 - theta) + theta * a_s
    speed = math.sqrt(theta * h * g * s / K)
    p = orc.Problem(rows, cols, l, z, theta, a_s, a_p, g=g, dt_max=0.05)
    m0 = p.mass(np.full(rows * cols, h))
    v10 = np.full(rows * cols, speed * math.cos(phi))
    v20 = np.full(rows * cols, speed * math.sin(phi))
    k = 8
    res = p.run(m0, v10, v20, 0.0, 1.0e9, max_steps=k)
    r = np.arange(rows)[:, None] + 0 * np.arange(cols)[None, :]
    c = 0 * r + np.arange(cols)[None, :]
    inner = ((r > k) & (r < rows - 1 - k) & (c > k) & (c < cols - 1 - k)).reshape(-1)
    assert inner.sum() >= 100
    assert np.abs(res["m"][inner] / m0[inner] - 1).max() <= 1e-12
    assert np.abs(res["v1"][inner] - v10[inner]).max() <= 1e-12 * speed
    assert np.abs(res["v2"][inner] - v20[inner]).max() <= 1e-12 * speed
    # and a wrong depth is not a fixed point
    res2 = p.run(m0 * 1.1, v10, v20, 0.0, 1.0e9, max_steps=2)
    assert np.abs(res2["v1"][inner] - v10[inner]).max() > 1e-6 * speed


def test_friction_closed_form(orc):
    """v = mu gamma solves alpha v + beta |v| v = gamma; beta = 0 gives gamma / alpha;
    alpha = 0 gives beta |v| v = gamma; alpha = beta = 0 gives v = 0 (Eq. miu-formula)."""
    rng = np.random.default_rng(11)
    for _ in range(2000):
        alpha = rng.choice([0.0, 10 ** rng.uniform(-6, 1)])
        beta = rng.choice([0.0, 10 ** rng.uniform(-6, 2)])
        g1, g2 = rng.normal(size=2) * 10 ** rng.uniform(-5, 0)
        v1, v2 = orc.friction(alpha, beta, g1, g2)
        nv = math.hypot(v1, v2)
        if alpha == 0.0 and beta == 0.0:
            assert v1 == 0.0 and v2 == 0.0
            continue
        r1 = alpha * v1 + beta * nv * v1 - g1
        r2 = alpha * v2 + beta * nv * v2 - g2
        assert math.hypot(r1, r2) <= 1e-13 * math.hypot(g1, g2)
        # v is parallel to gamma
        assert abs(v1 * g2 - v2 * g1) <= 1e-13 * nv * math.hypot(g1, g2) + 1e-300
    v1, v2 = orc.friction(2.0, 0.0, 3.0, -1.0)
    assert (v1, v2) == pytest.approx((1.5, -0.5), rel=1e-15)


def test_positivity_under_cfl(orc):
    """With CFL <= 1 the update keeps theta h >= 0 without clamping (Appendix A)."""
    sc = inputs.tiny(20, 18, seed=21, bc=(1, 0, 1, 0))
    p = orc.Problem(sc.rows, sc.cols, sc.l, sc.z, sc.theta, sc.alpha_s, sc.alpha_p, bc=sc.bc,
                    cfl=0.95, dt_max=100.0)
    h, v1, v2 = inputs.random_state(sc, 4, wet_fraction=0.5, depth=0.3, speed=2.0)
    res = p.run(p.mass(h), v1, v2, 0.0, 1.0e9, max_steps=300)
    assert res["ledger"].clamped == 0.0
    assert res["m"].min() >= 0.0


def test_stability_of_shallow_lake_under_cfl(orc):
    """A 2 mm lake with 30 % random surface noise, no friction, at CFL 0.95: the time step
    of Eqs. fvm_2D_eq_frac.12-13, where the gravity-wave speed sqrt(g h) dominates c_max,
    keeps the explicit scheme stable (velocities stay below 1 m/s, no clamping)."""
    rng = np.random.default_rng(1)
    p = orc.Problem(20, 18, 1.0, 0.0, 1.0, 0.0, 0.0, cfl=0.95, dt_max=100.0)
    h = 0.002 * (1 + 0.3 * rng.uniform(size=360))
    res = p.run(p.mass(h), 0.0, 0.0, 0.0, 1.0e9, max_steps=300)
    assert res["ledger"].clamped == 0.0 and res["m"].min() >= 0.0
    assert np.abs(res["v1"]).max() < 1.0 and np.abs(res["v2"]).max() < 1.0
    assert res["t"] > 100.0


def test_single_cell_rain_and_friction(orc):
    """One walled cell has no fluxes, so Eq. fvm_2D_eq_frac.07 reduces to
      theta h^{n+1} = theta h^n + dt M(t^{n+1})                       (rain at t^{n+1})
      theta h^{n+1} v^{n+1} = theta h^n v^n - dt K(h^{n+1}) |v^{n+1}| v^{n+1}.
    With a rain rate growing linearly in time the first line fixes the right-end
    quadrature; the second is checked as a residual with the new depth in K."""
    a = 1e-5                                    # r(t) = a t  [m/s]
    theta, a_s, a_p = 0.7, 0.01, 60.0
    p = orc.Problem(1, 1, 1.0, 0.0, theta, a_s, a_p, rain_t=[0.0, 1000.0], rain_r=[0.0, a * 1000.0])
    m, v1, v2 = np.array([0.05 * theta]), np.array([0.8]), np.array([-0.3])
    t = 10.0
    for dt in (0.5, 2.0, 7.0):
        mn, a1, b1 = p.step(m, v1, v2, dt, t + dt)
        assert mn[0] - m[0] == pytest.approx(dt * a * (t + dt), rel=1e-12)
        hn = mn[0] / theta
        K = a_p * hn * (1 - theta) + theta * a_s      # Eq. eq_K_h_theta at h^{n+1}
        nv = math.hypot(a1[0], b1[0])
        r1 = mn[0] * a1[0] - (m[0] * v1[0] - dt * K * nv * a1[0])
        r2 = mn[0] * b1[0] - (m[0] * v2[0] - dt * K * nv * b1[0])
        assert abs(r1) <= 1e-15 and abs(r2) <= 1e-15
        m, v1, v2, t = mn, a1, b1, t + dt


def test_phi_is_hexagon_area_over_perimeter(orc):
    """phi = sigma / (6 l): area by the shoelace formula over the six vertices of a
    pointy-top hexagon of circumradius l, divided by its perimeter."""
    for l in (0.5, 1.0, 41.0):
        ang = [math.radians(30 + 60 * k) for k in range(6)]
        vx = [l * math.cos(a) for a in ang]
        vy = [l * math.sin(a) for a in ang]
        area = 0.5 * abs(sum(vx[k] * vy[(k + 1) % 6] - vx[(k + 1) % 6] * vy[k] for k in range(6)))
        per = sum(math.hypot(vx[(k + 1) % 6] - vx[k], vy[(k + 1) % 6] - vy[k]) for k in range(6))
        assert orc.sigma(l) == pytest.approx(area, rel=1e-14)
        assert orc.phi(l) == pytest.approx(area / per, rel=1e-14)
        # neighbour centres sit at distance sqrt(3) l: the hexagons tile the raster
        x, y = _centres(3, 3, l)
        assert math.hypot(x[4] - x[5], y[4] - y[5]) == pytest.approx(math.sqrt(3) * l)
        assert math.hypot(x[4] - x[7], y[4] - y[7]) == pytest.approx(math.sqrt(3) * l)


def _golden_susita():
    rows, facts = [], {}
    with open(os.path.join(GOLDEN, "susita_volumes.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            if len(parts) == 4:
                rows.append(tuple(float(v) for v in parts))
            else:
                facts[parts[0]] = float(parts[1])
    return rows, facts


def test_susita_rain_volume(orc):
    """The printed rainfall volume of the Susita storm follows from the cell count and the
    radius with sigma = (3 sqrt3 / 2) l^2 and M = r(t) (the same for theta = 1 and 0.97),
    and the printed volumes satisfy rain - out = left."""
    table, facts = _golden_susita()
    for theta, rain, out, left in table:
        assert rain - out == left
    n_cells, l = int(facts["cells"]), facts["radius_m"]
    T_d, i_a, t_a = facts["T_d_s"], facts["i_a_mm_s"] * 1e-3, facts["t_a_s"]
    assert i_a * T_d / 2 == pytest.approx(facts["h0_m"], rel=1e-12)
    rt = np.array([0.0, t_a, T_d])
    rr = np.array([0.0, i_a, 0.0])
    vols = []
    for theta in (1.0, 0.97):
        p = orc.Problem(3, 4, l, 0.0, theta, 0.00709, 73.39, dt_max=0.25, rain_t=rt, rain_r=rr)
        res = p.run(np.zeros(12), 0.0, 0.0, 0.0, 3000.0)
        per_cell = res["ledger"].rain_in / 12
        vols.append(per_cell * n_cells)
        # walls and a flat bed: everything that fell is stored
        assert p.storage(res["m"]) == pytest.approx(res["ledger"].rain_in, rel=1e-12)
        assert p.storage(res["m"]) / (12 * p.sigma) == pytest.approx(facts["h0_m"], rel=1e-3)
    assert vols[0] == pytest.approx(vols[1], rel=1e-14)
    # the paper's radius is printed rounded to 41 m; the volume agrees to 0.3 %
    assert vols[0] == pytest.approx(table[0][1], rel=3e-3)


def test_two_cell_dam_break_by_hand(orc):
    """Two cells side by side (1 x 2 raster, walls, flat bed, theta = 1, no friction),
    depths 1 and 0.5, at rest.  Worked from the paper's equations:
      step 1: v_n = 0, so L = J = 0; w_0 > w_1 so the pressure mass is theta_0 h_0 = 1;
              each cell receives S_1 = -1/2 l (w_1 - w_0) * 1 * n_1 = g l / 4 (n = +x);
              gamma_1 = dt / sigma * g l / 4 and, with beta = 0, v = gamma / m:
              v_0 = dt g l / (4 sigma), v_1 = dt g l / (2 sigma), both towards the
              shallow cell; masses unchanged.
      step 2: v_n = (v_0 + v_1) / 2 > 0, so the upwind mass is theta_0 h_0 and cell 0
              loses dt l * 1 * v_n / sigma of depth to cell 1."""
    g, l, dt = 9.81, 1.0, 0.01
    sigma = 1.5 * math.sqrt(3.0) * l * l
    p = orc.Problem(1, 2, l, 0.0, 1.0, 0.0, 0.0, g=g)
    m1, a1, b1 = p.step(np.array([1.0, 0.5]), np.zeros(2), np.zeros(2), dt, dt)
    assert m1 == pytest.approx([1.0, 0.5], abs=0)
    assert a1 == pytest.approx([dt * g * l / (4 * sigma), dt * g * l / (2 * sigma)], rel=1e-14)
    assert np.abs(b1).max() == 0.0
    m2, a2, b2 = p.step(m1, a1, b1, dt, 2 * dt)
    vn = (a1[0] + a1[1]) / 2
    assert m2 == pytest.approx([1.0 - dt * l * vn / sigma, 0.5 + dt * l * vn / sigma], rel=1e-14)
    assert m2.sum() == pytest.approx(1.5, rel=1e-15)


def test_free_outflow_only(orc):
    """A free-discharge side lets water out but never in: under a uniform westward
    velocity the east column only loses water, the west column loses what leaves."""
    p = orc.Problem(4, 4, 1.0, 0.0, 1.0, 0.0, 0.0, bc=(1, 1, 1, 1))
    m = np.full(16, 0.1)
    res = p.run(m, -0.5, 0.0, 0.0, 1.0e9, max_steps=1)
    assert res["ledger"].outflow > 0
    east = [r * 4 + 3 for r in range(4)]
    west = [r * 4 for r in range(4)]
    assert (res["m"][east] < 0.1).all()
    assert (res["m"][west] <= 0.1 + 1e-15).all() and res["m"][west].sum() < 0.4
    assert p.storage(res["m"]) + res["ledger"].outflow == pytest.approx(p.storage(m), rel=1e-14)
    # the same field moving east through a walled west side: nothing leaves there
    q = orc.Problem(4, 4, 1.0, 0.0, 1.0, 0.0, 0.0, bc=(1, 0, 0, 0))
    res2 = q.run(m, 0.5, 0.0, 0.0, 1.0e9, max_steps=1)
    assert res2["ledger"].outflow == 0.0


# ----------------------------------------------------------------------------- artificial viscosity

def _two_cells(orc, hA, hB, vA, vB, viscosity, l=2.0, dt=0.01):
    """A 1 x 2 raster (walls all round, flat bed, no friction, no rain): one step."""
    p = orc.Problem(1, 2, l, np.zeros(2), np.ones(2), np.zeros(2), np.zeros(2), viscosity=viscosity,
                    dt_max=dt)
    m = np.array([hA, hB], dtype=np.float64)
    v1 = np.array([vA[0], vB[0]], dtype=np.float64)
    v2 = np.array([vA[1], vB[1]], dtype=np.float64)
    res = p.run(m, v1, v2, 0.0, dt, max_steps=1)
    return p, res


def test_viscosity_two_cells_closed_form(orc):
    """Appendix A, Eqs. eq_artif_visc and eq_visc1, worked by hand.  Two cells share an
    east-west edge (normal (1, 0)); both move along the edge (v = (0, v_2)), so v_n = 0: no
    mass moves, and the pressure term acts along the normal only.  With no friction the
    tangential velocity after one step is
      v_2A' = v_2A + dt / sigma * l c mu (v_2B - v_2A) / m_A,
    c = max(c_A, c_B), c = |v| + sqrt(g h), mu = 2 m_A m_B / (m_A + m_B)."""
    g, l, dt = 9.81, 2.0, 0.01
    hA, hB, vA, vB = 0.2, 0.1, (0.0, 0.3), (0.0, -0.1)
    p, off = _two_cells(orc, hA, hB, vA, vB, False, l, dt)
    assert off["v2"][0] == pytest.approx(vA[1], abs=1e-15)
    assert off["v2"][1] == pytest.approx(vB[1], abs=1e-15)
    p, on = _two_cells(orc, hA, hB, vA, vB, True, l, dt)
    sigma = 1.5 * math.sqrt(3.0) * l * l
    c = max(abs(vA[1]) + math.sqrt(g * hA), abs(vB[1]) + math.sqrt(g * hB))
    mu = 2.0 * hA * hB / (hA + hB)
    t = l * c * mu
    assert on["m"] == pytest.approx([hA, hB], abs=1e-15)
    assert on["v2"][0] == pytest.approx(vA[1] + dt / sigma * t * (vB[1] - vA[1]) / hA, rel=1e-13)
    assert on["v2"][1] == pytest.approx(vB[1] + dt / sigma * t * (vA[1] - vB[1]) / hB, rel=1e-13)
    # the normal component is the pressure term alone, as without viscosity (v_1 = 0)
    assert on["v1"] == pytest.approx(off["v1"], rel=1e-13)


def test_viscosity_conserves_momentum_and_dry_pairs(orc):
    """The viscous flux is antisymmetric: from the same state one step with and one
    without viscosity (same dt and masses, no friction) differ in total momentum
    sum(theta h v) only by rounding, although single velocities change; the field gets
    smoother than without viscosity; between two dry cells (0/0 := 0) nothing moves.
    (Total momentum itself is not conserved: the pressure term is the non-conservative
    g h grad w form of Eq. fvm_2D_eq_frac.01.)"""
    rng = np.random.default_rng(4)
    R, Cc, l = 12, 14, 1.0
    m = np.full(R * Cc, 0.8 * 0.05) * rng.uniform(0.5, 1.5, R * Cc)
    v1 = rng.uniform(-0.2, 0.2, R * Cc)
    v2 = rng.uniform(-0.2, 0.2, R * Cc)
    out = {}
    for visc in (False, True):
        p = orc.Problem(R, Cc, l, np.zeros(R * Cc), np.full(R * Cc, 0.8), np.zeros(R * Cc), np.zeros(R * Cc),
                        viscosity=visc, dt_max=0.002)
        one = p.run(m, v1, v2, 0.0, 1.0, max_steps=1)
        ten = p.run(m, v1, v2, 0.0, 1.0, max_steps=10)
        out[visc] = (one, ten)
    (o0, t0), (o1, t1) = out[False], out[True]
    assert o0["t"] == o1["t"] and np.array_equal(o0["m"], o1["m"])
    for k, a0 in (("v1", v1), ("v2", v2)):
        assert np.max(np.abs(o1[k] - o0[k])) > 1e-6
        assert abs(np.sum(o1["m"] * o1[k]) - np.sum(o0["m"] * o0[k])) <= 1e-14 * np.sum(m * np.abs(a0))
        assert np.std(t1[k]) < np.std(t0[k])
    _, dry = _two_cells(orc, 0.0, 0.0, (0.0, 0.3), (0.0, -0.1), True)
    assert np.all(np.isfinite(dry["v2"])) and np.all(dry["m"] == 0.0)


# ----------------------------------------------------------------------------- Thacker's problem

def test_thacker_exact_solution_transcription():
    """The analytic solution of Appendix B, as written in tests/thacker_exact.py, satisfies
    the continuity equation h_t + u h_x + v h_y = 0 (uniform velocity) in the wet region,
    and starts at rest under the stated plane (checked by central differences)."""
    import thacker_exact as TE
    T = inputs.THACKER
    x, y = np.array([480.0, 520.0, 500.0]), np.array([495.0, 505.0, 500.0])
    e = 1e-4
    for t in (1.0, 10.0, 30.0):
        u, v, _, h = TE.solution(T, t, x, y)
        assert np.all(h > 1.0)
        ht = (TE.solution(T, t + e, x, y)[3] - TE.solution(T, t - e, x, y)[3]) / (2 * e)
        hx = (TE.solution(T, t, x + e, y)[3] - TE.solution(T, t, x - e, y)[3]) / (2 * e)
        hy = (TE.solution(T, t, x, y + e)[3] - TE.solution(T, t, x, y - e)[3]) / (2 * e)
        assert np.max(np.abs(ht + u * hx + v * hy)) <= 1e-8
    u0, v0, w0, _ = TE.solution(T, 0.0, x, y)
    assert u0 == 0.0 and v0 == 0.0
    assert np.allclose(w0, 15.0 - 0.02 * (x - 500.0) + 0.1 * (y - 500.0), atol=1e-12)


def _thacker_run(orc, l):
    import thacker_exact as TE
    sc = inputs.thacker(l=l)
    p = orc.from_scenario(sc)
    res = p.run(p.mass(sc.h0), sc.v1_0, sc.v2_0, 0.0, 10.0)
    x, y = inputs.cell_centres(sc.rows, sc.cols, l)
    x, y = x + sc.meta["x_origin"], y + sc.meta["y_origin"]
    u, v, w, h = TE.solution(inputs.THACKER, 10.0, x, y)
    m = res["m"].reshape(sc.rows, sc.cols)
    wet = h > 0.1
    return dict(l1=float(np.abs(m - h).sum() / h.sum()),
                u=float(res["v1"].reshape(h.shape)[wet].mean()), v=float(res["v2"].reshape(h.shape)[wet].mean()),
                u_ex=float(u), v_ex=float(v))


def test_thacker_oracle_converges_to_analytic(orc):
    """Thacker's problem (Sec. 4, Appendix B): with the linear resistance -tau h v the
    oracle approaches the analytic solution at first order.  At t = 10 s the relative L1
    depth error roughly halves from l = 4 m to l = 2 m, and the mean velocity of the wet
    region matches the analytic uniform velocity."""
    c, f = _thacker_run(orc, 4.0), _thacker_run(orc, 2.0)
    assert c["l1"] <= 0.03 and f["l1"] <= 0.015
    assert f["l1"] <= 0.6 * c["l1"]
    assert f["u"] == pytest.approx(f["u_ex"], rel=0.03)
    assert f["v"] == pytest.approx(f["v_ex"], rel=0.06)


# ----------------------------------------------------------------------------- given mass flux, Dirichlet

def _flux_problem(orc, rows, cols, l, q, z=None, h0=0.1, alpha_s=0.0, east=0):
    n = rows * cols
    zz = np.zeros(n) if z is None else z
    p = orc.Problem(rows, cols, l, zz, np.ones(n), np.full(n, alpha_s), np.zeros(n), bc=(2, east, 0, 0),
                    bc_q=(q, 0.0, 0.0, 0.0), dt_max=0.05)
    return p, np.full(n, h0)


def test_flux_boundary_inflow_by_hand(orc):
    """Given mass flux q on the west side (Sec. 3): the edges on that side admit
    l q (n_side . n_edge).  On 4 rows: every row's west edge (4 l) plus, for the even
    rows 0 and 2, the NW / SW edges that leave the raster through the west side
    (row 0: NW only, its SW leaves through the south side; row 2: both), each l / 2:
    5.5 l in all.  One step from a lake at rest gains exactly dt q 5.5 l, and the ledger
    books it as negative outflow."""
    l, q = 1.0, 0.02
    p, h = _flux_problem(orc, 4, 3, l, q)
    m = p.mass(h)
    res = p.run(m, np.zeros(12), np.zeros(12), 0.0, 0.05, max_steps=1)
    dt = res["t"]
    gain = (np.sum(res["m"]) - np.sum(m)) * p.sigma
    assert gain == pytest.approx(dt * q * 5.5 * l, rel=1e-12)
    led = res["ledger"]
    assert led.outflow == pytest.approx(-dt * q * 5.5 * l, rel=1e-12)
    # the inflow carries momentum east at q / h (h = 0.1 m above the critical depth): from
    # rest, with no friction and no pressure term yet, v_1 = dt / sigma q_in (q / h) / m'
    v1 = res["v1"].reshape(4, 3)
    mn = res["m"].reshape(4, 3)
    for r, share in ((1, 1.0), (2, 2.0), (3, 1.0)):
        qin = l * q * share
        assert v1[r, 0] == pytest.approx(dt / p.sigma * qin * (q / 0.1) / mn[r, 0], rel=1e-12)
    assert np.max(np.abs(res["v2"])) <= 1e-12 * np.abs(v1).max()


def test_flux_boundary_reaches_normal_depth(orc):
    """A sloping channel (s = 1 %) fed by q = 0.01 m^2/s through its west side, free at
    the east end, soil friction only: the flow settles to the uniform normal depth of
    the friction balance alpha_s v^2 = g s h with v h = q, h_n = (alpha_s q^2 / (g s))^(1/3),
    in the middle of the channel (Eqs. eq_tsa_darcy, fvm_2D_eq_frac.07 in steady state)."""
    rows, cols, l, q, s, a_s, g = 12, 60, 1.0, 0.01, 0.01, 0.00709, 9.81
    x, _ = inputs.cell_centres(rows, cols, l)
    z = (s * (x.max() - x)).ravel()
    hn = (a_s * q * q / (g * s)) ** (1.0 / 3.0)
    p, h = _flux_problem(orc, rows, cols, l, q, z=z, h0=hn, alpha_s=a_s, east=1)
    m = p.mass(h)
    res = p.run(m, np.full(rows * cols, q / hn), np.zeros(rows * cols), 0.0, 300.0)
    hm = res["m"].reshape(rows, cols)
    mid = hm[rows // 2 - 1:rows // 2 + 1, cols // 3:2 * cols // 3]
    qm = (res["m"] * res["v1"]).reshape(rows, cols)[rows // 2 - 1:rows // 2 + 1, cols // 3:2 * cols // 3]
    assert np.mean(mid) == pytest.approx(hn, rel=0.03)
    assert np.mean(qm) == pytest.approx(q, rel=0.03)
    # steady: the outflow through the east side equals the inflow
    p2 = orc.Problem(rows, cols, l, z, np.ones(rows * cols), np.full(rows * cols, a_s), np.zeros(rows * cols),
                     bc=(2, 1, 0, 0), bc_q=(q, 0, 0, 0), dt_max=0.05)
    one = p2.run(res["m"], res["v1"], res["v2"], 0.0, 10.0)
    inflow_rate = q * (rows * 1.5 * l)            # projected west side, about 1.5 l per row
    # over 10 more seconds storage hardly changes: net boundary flow ~ 0 against 10 s of inflow
    assert abs(np.sum(one["m"]) - np.sum(res["m"])) * p2.sigma <= 0.02 * inflow_rate * 10.0
    assert abs(one["ledger"].outflow) <= 0.02 * inflow_rate * 10.0


def test_dirichlet_boundary_rest_and_inflow(orc):
    """Dirichlet side (Sec. 4, Eq. numerics-bc): a ghost at the lake's own level and at
    rest leaves the lake exactly at rest; a higher ghost level drives water in, and the
    ledger books the inflow (storage gain = -outflow, no rain)."""
    rows, cols, l = 6, 8, 1.0
    n = rows * cols
    for hb, moves in ((0.1, False), (0.15, True)):
        p = orc.Problem(rows, cols, l, np.zeros(n), np.ones(n), np.zeros(n), np.zeros(n), bc=(3, 0, 0, 0),
                        bc_h=(hb, 0, 0, 0), bc_u=(0.0, 0, 0, 0), dt_max=0.02)
        m = p.mass(np.full(n, 0.1))
        res = p.run(m, np.zeros(n), np.zeros(n), 0.0, 0.4)
        led = res["ledger"]
        if not moves:
            assert np.max(np.abs(res["m"] - m)) == 0.0 and np.max(np.abs(res["v1"])) == 0.0
        else:
            gain = (np.sum(res["m"]) - np.sum(m)) * p.sigma
            assert gain > 0 and gain == pytest.approx(-led.outflow, rel=1e-12)
            assert np.all(res["v1"].reshape(rows, cols)[:, 0] > 0.0)
