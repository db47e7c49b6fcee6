"""Seeded synthetic inputs for the hexagonal porous Saint-Venant solver.

This module builds terrains, porosity / land-cover maps and storms of the shapes the
paper's hillslope and catchment cases use (a planar vegetated slope, a fractal basin
with vegetation patches, an ensemble of hillslopes, a large carved catchment).  The
paper's own DEMs and flume data are not available; every field here is synthetic and
reproducible from its seed.

It holds no arithmetic of the flow scheme itself: it only produces inputs (bed
elevation, porosity, coefficients, initial state, hyetograph tables, boundary types)
that both the CUDA path and the CPU oracle consume.

Conventions shared with the solver's interface:
  * raster of ``rows x cols`` pointy-top hexagons, row-major, odd rows shifted east by
    half a centre spacing; edge length ``l``; cell centre of (r, c) at
    x = sqrt(3) l (c + (r odd)/2), y = 1.5 l r;
  * elevations are float32 values (the solver stores the bed in float32; the oracle
    reads the same values in double);
  * boundary type per side in the order W, E, S, N (0 = wall, 1 = free discharge),
    with an optional [begin, end) interval along a side where free discharge applies;
  * hyetographs are piecewise-linear tables (t [s], r [m/s]), zero outside the table.
"""
from __future__ import annotations

import heapq
import math
from dataclasses import dataclass, field

import numpy as np

MM_PER_H = 1.0e-3 / 3600.0          # 1 mm/h in m/s
WALL, FREE, FLUX, DIRICHLET = 0, 1, 2, 3
ALPHA_S_DEFAULT = 0.00709           # soil friction coefficient fitted in the flume study (Sec. 4.3)
ALPHA_P_DEFAULT = 73.39             # plant drag coefficient fitted in the flume study (Sec. 4.3)


@dataclass
class Scenario:
    """One raster's inputs.  ``theta`` or (``cls`` + class tables) describe porosity."""
    name: str
    rows: int
    cols: int
    l: float
    z: np.ndarray                      # float32 (rows, cols)
    theta: np.ndarray                  # float32 (rows, cols)
    alpha_s: np.ndarray                # float32 (rows, cols)
    alpha_p: np.ndarray                # float32 (rows, cols)
    h0: np.ndarray                     # float32 (rows, cols)
    v1_0: np.ndarray                   # float32 (rows, cols)
    v2_0: np.ndarray                   # float32 (rows, cols)
    bc: tuple = (WALL, WALL, WALL, WALL)
    free_range: tuple = ((0, 0), (0, 0), (0, 0), (0, 0))   # (0, 0) = whole side
    rain_t: np.ndarray = field(default_factory=lambda: np.zeros(0))
    rain_r: np.ndarray = field(default_factory=lambda: np.zeros(0))
    t_end: float = 0.0
    g: float = 9.81
    cfl: float = 0.5
    dt_max: float = 1.0
    sample_dt: float = 0.0
    cls: np.ndarray | None = None      # uint8 (rows, cols) land-cover class, optional
    class_theta: np.ndarray | None = None
    class_alpha_p: np.ndarray | None = None
    class_alpha_s: np.ndarray | None = None
    meta: dict = field(default_factory=dict)
    viscosity: bool = False            # artificial viscosity on (Appendix A, Eq. eq_artif_visc)
    tau: float = 0.0                   # linear soil resistance -tau h v [1/s] (Thacker's problem)
    h_dry: float = 0.0                 # depth below which velocities are zeroed [m] (0 = none)
    bc_q: tuple = (0.0, 0.0, 0.0, 0.0)  # FLUX sides: inflow per unit length [m^2/s]
    bc_h: tuple = (0.0, 0.0, 0.0, 0.0)  # DIRICHLET sides: ghost depth [m]
    bc_u: tuple = (0.0, 0.0, 0.0, 0.0)  # DIRICHLET sides: ghost speed along the inward normal [m/s]

    @property
    def n(self) -> int:
        return self.rows * self.cols


# ----------------------------------------------------------------------------- geometry

def cell_centres(rows: int, cols: int, l: float):
    """Centre coordinates (x, y) [m] of every cell, each (rows, cols) float64."""
    r = np.arange(rows, dtype=np.float64)[:, None]
    c = np.arange(cols, dtype=np.float64)[None, :]
    x = math.sqrt(3.0) * l * (c + 0.5 * (r.astype(np.int64) & 1))
    y = 1.5 * l * r + 0.0 * c
    return x + 0.0 * r, y


# ----------------------------------------------------------------------------- random fields

def fbm(rows: int, cols: int, hurst: float, rms: float, rng: np.random.Generator,
        dx: float = 1.0, dy: float = 1.0) -> np.ndarray:
    """Fractional-Brownian surface by spectral synthesis: amplitude ~ k^-(H+1), zero mean,
    scaled to the given RMS.  (rows, cols) float64."""
    ky = np.fft.fftfreq(rows, d=dy)[:, None]
    kx = np.fft.rfftfreq(cols, d=dx)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    k[0, 0] = 1.0
    amp = k ** (-(hurst + 1.0))
    amp[0, 0] = 0.0
    ph = rng.uniform(0.0, 2.0 * np.pi, size=amp.shape)
    spec = amp * np.exp(1j * ph) * rng.standard_normal(size=amp.shape)
    f = np.fft.irfft2(spec, s=(rows, cols))
    f -= f.mean()
    s = f.std()
    return f * (rms / s if s > 0 else 0.0)


def grf(rows: int, cols: int, corr_cells: float, rng: np.random.Generator) -> np.ndarray:
    """Gaussian random field: white noise smoothed with a Gaussian of the given width,
    standardised to zero mean and unit variance."""
    from scipy.ndimage import gaussian_filter
    f = gaussian_filter(rng.standard_normal((rows, cols)), sigma=corr_cells, mode="wrap")
    f -= f.mean()
    s = f.std()
    return f / s if s > 0 else f


# ----------------------------------------------------------------------------- storms

def constant_rain(rate_mm_h: float, duration_s: float, start_s: float = 0.0):
    return (np.array([start_s, start_s + duration_s]),
            np.array([rate_mm_h, rate_mm_h]) * MM_PER_H)


def triangular_rain(total_s: float, peak_s: float, peak_mm_h: float):
    """Triangular hyetograph of Appendix C: 0 -> i_a at t_a -> 0 at T_d."""
    return (np.array([0.0, peak_s, total_s]), np.array([0.0, peak_mm_h, 0.0]) * MM_PER_H)


def table_rain(points_min_mm_h):
    t = np.array([p[0] * 60.0 for p in points_min_mm_h])
    r = np.array([p[1] for p in points_min_mm_h]) * MM_PER_H
    return t, r


# ----------------------------------------------------------------------------- scenarios

def _fill(shape, v, dtype=np.float32):
    return np.full(shape, v, dtype=dtype)


def hillslope(rows=64, cols=64, l=1.0, slope=0.05, theta=0.9, rain_mm_h=50.0, rain_s=600.0,
              t_end=600.0, alpha_s=ALPHA_S_DEFAULT, alpha_p=ALPHA_P_DEFAULT) -> Scenario:
    """Planar vegetated hillslope: bed falling along x at `slope`, uniform porosity, dry
    start, constant rain, free discharge at the downslope (east) side, walls elsewhere.
    Defaults: 64 x 64 cells, edge 1 m, 5 % slope, porosity 0.9, 50 mm/h for 600 s."""
    x, _ = cell_centres(rows, cols, l)
    z = (slope * (x.max() - x)).astype(np.float32)
    sh = (rows, cols)
    rt, rr = constant_rain(rain_mm_h, rain_s)
    return Scenario("hillslope", rows, cols, l, z, _fill(sh, theta), _fill(sh, alpha_s),
                    _fill(sh, alpha_p), _fill(sh, 0.0), _fill(sh, 0.0), _fill(sh, 0.0),
                    bc=(WALL, FREE, WALL, WALL), rain_t=rt, rain_r=rr, t_end=t_end)


def fractal_basin(rows=1024, cols=1024, l=2.0, seed=1002, hurst=0.8, rms=10.0, tilt=0.10,
                  cover=0.40, corr_cells=20.0, theta_lo=0.7, theta_hi=0.95, storm_s=3600.0,
                  peak_s=1800.0, peak_mm_h=100.0, t_end=3600.0) -> Scenario:
    """fBm terrain (Hurst 0.8) plus a mean tilt along x, vegetation patches from a
    thresholded Gaussian random field covering `cover` of the cells with porosity mapped
    linearly into [theta_lo, theta_hi] (1.0 outside), triangular storm, free discharge
    on every side (the paper's default boundary)."""
    rng = np.random.default_rng(seed)
    x, y = cell_centres(rows, cols, l)
    z = fbm(rows, cols, hurst, rms, rng, dx=math.sqrt(3) * l, dy=1.5 * l)
    z = z + tilt * (x.max() - x)
    z -= z.min()
    f = grf(rows, cols, corr_cells, rng)
    thr = np.quantile(f, 1.0 - cover)
    patch = f >= thr
    fmax = f.max()
    frac = np.clip((f - thr) / max(fmax - thr, 1e-12), 0.0, 1.0)
    theta = np.where(patch, theta_hi - (theta_hi - theta_lo) * frac, 1.0).astype(np.float32)
    sh = (rows, cols)
    rt, rr = triangular_rain(storm_s, peak_s, peak_mm_h)
    return Scenario("fractal_basin", rows, cols, l, z.astype(np.float32), theta,
                    _fill(sh, ALPHA_S_DEFAULT), _fill(sh, ALPHA_P_DEFAULT), _fill(sh, 0.0),
                    _fill(sh, 0.0), _fill(sh, 0.0), bc=(FREE, FREE, FREE, FREE), rain_t=rt,
                    rain_r=rr, t_end=t_end, meta=dict(seed=seed, cover=float(patch.mean())))


def _member_draws(rng: np.random.Generator, n_lo: int, n_hi: int, n_override: int | None) -> dict:
    u = rng.uniform()
    n = int(round(n_lo * (n_hi / n_lo) ** u)) if n_override is None else int(n_override)
    return dict(n=n, slope=rng.uniform(0.02, 0.30), cover=rng.uniform(0.0, 0.80),
                theta=rng.uniform(0.70, 0.95), alpha_p=rng.uniform(20.0, 100.0),
                rain_mm_h=rng.uniform(10.0, 150.0), rain_s=rng.uniform(20.0, 60.0) * 60.0)


def member_params(s: int, base_seed=3000, n_lo=128, n_hi=512, n_override: int | None = None) -> dict:
    """The scalar draws of ensemble member `s` (side n, slope, cover, porosity, drag, rain
    rate and duration) without building its fields."""
    return _member_draws(np.random.default_rng(base_seed + s), n_lo, n_hi, n_override)


def ensemble_member(s: int, base_seed=3000, n_lo=128, n_hi=512, l=2.0, t_end=6400.0,
                    n_override: int | None = None, corr_cells: float = 8.0) -> Scenario:
    """Member `s` of the hillslope ensemble: square raster with side drawn log-uniform in
    [n_lo, n_hi], planar slope 2-30 % falling along x, vegetation cover 0-80 % from a
    thresholded Gaussian random field, porosity in [0.7, 0.95] and plant drag in
    [20, 100] 1/m drawn per member, block rain of 10-150 mm/h lasting 20-60 min, free
    discharge downslope (east), walls elsewhere.  The cover field's correlation length
    is corr_cells cells."""
    rng = np.random.default_rng(base_seed + s)
    d = _member_draws(rng, n_lo, n_hi, n_override)
    n, slope, cover, theta_v = d["n"], d["slope"], d["cover"], d["theta"]
    alpha_p, rate, dur = d["alpha_p"], d["rain_mm_h"], d["rain_s"]
    x, _ = cell_centres(n, n, l)
    z = slope * (x.max() - x)
    if cover > 0:
        f = grf(n, n, corr_cells, rng)
        veg = f >= np.quantile(f, 1.0 - cover)
    else:
        veg = np.zeros((n, n), dtype=bool)
    theta = np.where(veg, theta_v, 1.0).astype(np.float32)
    sh = (n, n)
    rt, rr = constant_rain(rate, dur)
    return Scenario(f"member{s}", n, n, l, z.astype(np.float32), theta, _fill(sh, ALPHA_S_DEFAULT),
                    _fill(sh, alpha_p), _fill(sh, 0.0), _fill(sh, 0.0), _fill(sh, 0.0),
                    bc=(WALL, FREE, WALL, WALL), rain_t=rt, rain_r=rr, t_end=t_end,
                    meta=dict(seed=base_seed + s, slope=slope, cover=cover, theta=theta_v,
                              alpha_p=alpha_p, rain_mm_h=rate, rain_s=dur))


def _priority_flood_tree(zc: np.ndarray, outlet: tuple[int, int], eps: float):
    """Drainage tree of a coarse grid by priority flood from `outlet` (4-neighbour
    graph): returns (parent index or -1, filled elevation, flood order)."""
    R, Cc = zc.shape
    n = R * Cc
    parent = np.full(n, -1, dtype=np.int64)
    filled = np.full(n, np.inf)
    seen = np.zeros(n, dtype=bool)
    o = outlet[0] * Cc + outlet[1]
    filled[o] = zc.flat[o]
    seen[o] = True
    heap = [(filled[o], o)]
    order = []
    while heap:
        e, i = heapq.heappop(heap)
        order.append(i)
        r, c = divmod(i, Cc)
        for rr, cc in ((r + 1, c), (r - 1, c), (r, c + 1), (r, c - 1)):
            if 0 <= rr < R and 0 <= cc < Cc:
                j = rr * Cc + cc
                if not seen[j]:
                    seen[j] = True
                    filled[j] = max(zc.flat[j], e + eps)
                    parent[j] = i
                    heapq.heappush(heap, (filled[j], j))
    return parent, filled, np.array(order)


def carved_catchment(rows=4096, cols=4096, l=5.0, seed=1004, hurst=0.8, rms=50.0,
                     mean_slope=0.01, block=32, min_acc=12, outlet_halfwidth=2,
                     start_mm_h=None) -> Scenario:
    """Large catchment: fBm relief (RMS 50 m) on a 1 % mean slope towards the south, a
    channel network carved along the drainage tree of a coarse priority flood so that the
    network reaches one outlet on the south side, land cover 50 / 30 / 20 % forest /
    grass / bare from Gaussian-random-field quantiles with per-class porosity and plant
    drag, and a 2 h double-peak storm (80 and 120 mm/h).  Only the outlet cells of the
    south side discharge freely; every other side is a wall.  Outlet discharge is sampled
    every 10 s."""
    rng = np.random.default_rng(seed)
    x, y = cell_centres(rows, cols, l)
    z = fbm(rows, cols, hurst, rms, rng, dx=math.sqrt(3) * l, dy=1.5 * l)
    z = z + mean_slope * y
    # coarse drainage tree
    R, Cc = rows // block, cols // block
    zc = z[:R * block, :Cc * block].reshape(R, block, Cc, block).mean(axis=(1, 3))
    out_c = Cc // 2
    parent, filled, order = _priority_flood_tree(zc, (0, out_c), eps=0.05 * block * l * 1e-2)
    acc = np.ones(R * Cc)
    for i in order[::-1]:
        if parent[i] >= 0:
            acc[parent[i]] += acc[i]
    # carve: channel bed descends along the tree; valleys widen with a bank slope
    bed = np.full((rows, cols), np.inf)
    depth = 2.0 * np.log1p(acc)
    bed_c = filled - depth
    for i in range(R * Cc):
        if acc[i] < min_acc:
            continue
        p = parent[i]
        r0, c0 = divmod(i, Cc)
        if p >= 0:
            r1, c1 = divmod(int(p), Cc)
            b0, b1 = bed_c[i], bed_c[p]
        else:
            r1, c1, b0, b1 = -0.5, c0, bed_c[i], bed_c[i] - 1.0
        nseg = 2 * block
        ts = np.linspace(0.0, 1.0, nseg + 1)
        rr = np.clip(((r0 + 0.5) + ts * (r1 - r0)) * block, 0, rows - 1).astype(np.int64)
        cc = np.clip(((c0 + 0.5) + ts * (c1 - c0)) * block, 0, cols - 1).astype(np.int64)
        bb = b0 + ts * (b1 - b0)
        np.minimum.at(bed, (rr, cc), bb)
    bank = 0.05 * l
    for _ in range(24):
        b = bed.copy()
        np.minimum(b[1:, :], bed[:-1, :] + bank, out=b[1:, :])
        np.minimum(b[:-1, :], bed[1:, :] + bank, out=b[:-1, :])
        np.minimum(b[:, 1:], bed[:, :-1] + bank, out=b[:, 1:])
        np.minimum(b[:, :-1], bed[:, 1:] + bank, out=b[:, :-1])
        bed = b
    z = np.minimum(z, bed)
    z -= z.min()
    # land cover classes from GRF quantiles: 0 forest 50 %, 1 grass 30 %, 2 bare 20 %
    f = grf(rows, cols, 40.0, rng)
    q50, q80 = np.quantile(f, [0.5, 0.8])
    cls = np.where(f < q50, 0, np.where(f < q80, 1, 2)).astype(np.uint8)
    class_theta = np.array([0.90, 0.97, 1.00], dtype=np.float32)
    class_alpha_p = np.array([80.0, 40.0, 0.0], dtype=np.float32)
    class_alpha_s = np.array([ALPHA_S_DEFAULT] * 3, dtype=np.float32)
    theta = class_theta[cls]
    sh = (rows, cols)
    c_out = int(out_c * block + block // 2)
    rt, rr = table_rain([(0, 0), (30, 80), (60, 20), (90, 120), (120, 0)])
    h0 = _fill(sh, 0.0)
    return Scenario("carved_catchment", rows, cols, l, z.astype(np.float32), theta,
                    class_alpha_s[cls], class_alpha_p[cls], h0, _fill(sh, 0.0), _fill(sh, 0.0),
                    bc=(WALL, WALL, FREE, WALL),
                    free_range=((0, 0), (0, 0), (c_out - outlet_halfwidth, c_out + outlet_halfwidth + 1),
                                (0, 0)),
                    rain_t=rt, rain_r=rr, t_end=7200.0, sample_dt=10.0, cls=cls,
                    class_theta=class_theta, class_alpha_p=class_alpha_p,
                    class_alpha_s=class_alpha_s, meta=dict(seed=seed, outlet_col=c_out))


def random_state(sc: Scenario, seed: int, wet_fraction=0.7, depth=0.05, speed=0.5):
    """Random wet/dry initial state for parity tests: depth drawn in [0, depth] on a random
    `wet_fraction` of the cells (0 elsewhere), velocities in [-speed, speed]."""
    rng = np.random.default_rng(seed)
    sh = (sc.rows, sc.cols)
    wet = rng.uniform(size=sh) < wet_fraction
    h = np.where(wet, rng.uniform(0.0, depth, size=sh), 0.0).astype(np.float32)
    v1 = rng.uniform(-speed, speed, size=sh).astype(np.float32)
    v2 = rng.uniform(-speed, speed, size=sh).astype(np.float32)
    return h, v1, v2


def tiny(rows, cols, seed, l=1.0, bc=(WALL, WALL, WALL, WALL), relief=0.2, theta_lo=0.6,
         rain_mm_h=0.0, smooth=False) -> Scenario:
    """Small random raster for parity tests: random bed (independent per cell, or a smooth
    fBm surface with `smooth`), random porosity per cell in [theta_lo, 1], random (uniform)
    friction and drag coefficients, random wet/dry state."""
    rng = np.random.default_rng(seed)
    sh = (rows, cols)
    if smooth:
        z = fbm(rows, cols, 0.8, relief, rng, dx=math.sqrt(3) * l, dy=1.5 * l)
        z = (z - z.min()).astype(np.float32)
    else:
        z = (relief * rng.uniform(size=sh)).astype(np.float32)
    theta = rng.uniform(theta_lo, 1.0, size=sh).astype(np.float32)
    a_s = np.full(sh, rng.uniform(0.0, 0.02), dtype=np.float32)
    a_p = np.full(sh, rng.uniform(0.0, 100.0), dtype=np.float32)
    sc = Scenario(f"tiny{rows}x{cols}", rows, cols, l, z, theta, a_s, a_p, _fill(sh, 0.0),
                  _fill(sh, 0.0), _fill(sh, 0.0), bc=tuple(bc))
    h, v1, v2 = random_state(sc, seed + 1)
    sc.h0, sc.v1_0, sc.v2_0 = h, v1, v2
    if rain_mm_h > 0:
        sc.rain_t, sc.rain_r = constant_rain(rain_mm_h, 1.0e6)
    return sc


THACKER = dict(a=1.25e-3, b=5.0e-3, x0=500.0, y0=500.0, tau=0.7, w0=15.0, du0=0.02 * 9.81, dv0=-0.1 * 9.81,
               g=9.81)


def thacker(l=1.0, x_range=(250.0, 750.0), y_range=(350.0, 650.0), t_end=10.0) -> Scenario:
    """Thacker's problem in its non-oscillating form (Sec. 4, Appendix B): paraboloid bed
    z = a (x - x0)^2 + b (y - y0)^2 (a = 1.25e-3, b = 5e-3 1/m, x0 = y0 = 500 m), no
    vegetation (theta = 1) and no rain, linear soil resistance -tau h v (tau = 0.7 1/s)
    and no other friction; at rest at t = 0 under the planar free surface
    w = 15 - 0.02 (x - x0) + 0.1 (y - y0) m (u'(0) = 0.02 g, v'(0) = -0.1 g).  The raster
    covers x_range x y_range (the water stays within about 110 m x 55 m of the centre,
    where the bed is far below the walls of the window); cells of edge l.  Velocities of
    cells shallower than 1 mm are set to zero (h_dry): with no resistance but the linear
    one, films at the moving shoreline otherwise accelerate without bound.  Courant number
    0.25: at 0.5 the still, 15 m deep centre of the bowl develops a growing mode after
    ~3,000 steps on the paper's mesh (in the FP64 oracle as on the GPU)."""
    T = THACKER
    cols = int(round((x_range[1] - x_range[0]) / (math.sqrt(3.0) * l)))
    rows = int(round((y_range[1] - y_range[0]) / (1.5 * l)))
    x, y = cell_centres(rows, cols, l)
    x = x + x_range[0]
    y = y + y_range[0]
    z = T["a"] * (x - T["x0"]) ** 2 + T["b"] * (y - T["y0"]) ** 2
    w = T["w0"] - (x - T["x0"]) * T["du0"] / T["g"] - (y - T["y0"]) * T["dv0"] / T["g"]
    sh = (rows, cols)
    z32 = z.astype(np.float32)
    h0 = np.maximum(w - z32.astype(np.float64), 0.0).astype(np.float32)
    sc = Scenario(f"thacker_l{l:g}", rows, cols, l, z32, _fill(sh, 1.0), _fill(sh, 0.0), _fill(sh, 0.0), h0,
                  _fill(sh, 0.0), _fill(sh, 0.0), bc=(WALL, WALL, WALL, WALL), t_end=t_end, g=T["g"],
                  meta=dict(T, x_origin=x_range[0], y_origin=y_range[0]))
    sc.tau = T["tau"]
    sc.h_dry = 1.0e-3
    sc.cfl = 0.25
    return sc


# ----------------------------------------------------------------------------- flume

# The vegetated flume of Sec. 4.2.2: 18 m x 1 m, bed slope 1.05 mm/m, emergent cylinders of
# radius 5 mm at 81 per m^2 over one half (theta_v = 1 - N pi R_c^2), upstream discharges of
# the six experiments in m^3/s (layout theta_1: vegetation on x >= 9 m; theta_2: on x < 9 m).
FLUME = dict(length=18.0, width=1.0, slope=1.05e-3, theta_v=1.0 - 81.0 * math.pi * 0.005 ** 2,
             q=((1, 0.007), (1, 0.015), (1, 0.021), (2, 0.007), (2, 0.015), (2, 0.050)))


def flume(q_l: float, layout: int, alpha_s: float = ALPHA_S_DEFAULT, alpha_p: float = ALPHA_P_DEFAULT,
          l: float = 0.1, tailwater: float = 0.1, t_end: float = 600.0, theta_v: float | None = None,
          slope: float | None = None) -> Scenario:
    """The flume of Sec. 4.2.2 on a hexagonal raster of edge l: bed z = m (18 - x), porosity
    theta_1 (layout 1) or theta_2 (layout 2), uniform soil friction alpha_s and plant drag
    alpha_p; theta_v and slope override the flume's vegetation porosity and bed slope (the
    environment of the sensitivity study).  The upstream (west) side admits the discharge
    q_l [m^3/s] as a given mass flux
    spread over the side's width (west_width); the downstream (east) side is a Dirichlet side
    at the tailwater depth, its ghost carrying the same discharge out (a tailgate: the
    zero-gradient outlet of the paper leaves a subcritical flow without control, and the
    depths do not settle); north and south are walls.  Initially at rest at the tailwater
    level over the bed."""
    F = FLUME
    theta_v = F["theta_v"] if theta_v is None else theta_v
    slope = F["slope"] if slope is None else slope
    cols = int(round(F["length"] / (math.sqrt(3.0) * l)))
    rows = max(2, int(round(F["width"] / (1.5 * l))))
    x, _ = cell_centres(rows, cols, l)
    sh = (rows, cols)
    z = (slope * (F["length"] - x)).astype(np.float32)
    veg = (x >= 9.0) if layout == 1 else (x < 9.0)
    theta = np.where(veg, theta_v, 1.0).astype(np.float32)
    level = tailwater + float(z.min())
    h0 = np.maximum(level - z.astype(np.float64), 0.0).astype(np.float32)
    q_side = q_l / west_width(rows, l)              # per unit width of the inflow side
    sc = Scenario(f"flume_q{q_l * 1e3:g}_t{layout}", rows, cols, l, z, theta, _fill(sh, alpha_s),
                  _fill(sh, alpha_p), h0, _fill(sh, 0.0), _fill(sh, 0.0), bc=(FLUX, DIRICHLET, WALL, WALL),
                  t_end=t_end, meta=dict(q_l=q_l, layout=layout, tailwater=tailwater, theta_v=theta_v,
                                         slope=slope))
    sc.bc_q = (q_side, 0.0, 0.0, 0.0)
    sc.bc_h = (0.0, tailwater, 0.0, 0.0)
    sc.bc_u = (0.0, -q_side / tailwater, 0.0, 0.0)
    return sc


def west_width(rows: int, l: float) -> float:
    """Width of a raster's west side seen by a flux along its normal: the sum over its
    boundary edges of l (n_W . n_edge).  Every row has its W edge (1); an even row, not
    shifted, also has its NW and SW edges on the side (1/2 each) when the neighbour row
    exists (else the edge belongs to the N or S side)."""
    even = [r for r in range(rows) if r % 2 == 0]
    return l * (rows + 0.5 * sum(1 for r in even if r + 1 < rows) + 0.5 * sum(1 for r in even if r >= 1))


def flume_gauges(sc: Scenario, n: int = 17) -> np.ndarray:
    """Flat indices of n gauges on the flume's centre row, evenly spaced from x = 0.5 m to
    x = 17.5 m (nearest cell centre)."""
    x, _ = cell_centres(sc.rows, sc.cols, sc.l)
    r = sc.rows // 2
    xs = np.linspace(0.5, FLUME["length"] - 0.5, n)
    cols = np.abs(x[r][None, :] - xs[:, None]).argmin(axis=1)
    return r * sc.cols + cols
