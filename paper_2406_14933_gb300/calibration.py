"""Sensitivity of the vegetated flume to the friction coefficients and their estimation
by pattern search (Sec. 4.3), run on the batched ensemble.

The flume of Sec. 4.2.2 (``inputs.flume``): 18 m x 1 m, bed slope 1.05 mm/m, vegetation
on one half, a given discharge through the upstream side and a tailwater depth held at
the downstream side, the artificial viscosity of Appendix A on (without it the scheme's
flume keeps sloshing; with it the depths settle geometrically), run to a steady state.

* ``h_bar``: the mean depth over the cells with x >= 9 m (Eq. eq_h_bar);
* ``sensitivity``: delta_s and delta_p, the averaged forward differences of h_bar over a
  regular (alpha_s, alpha_p) grid (Sec. 4.3); ``sensitivity_sweep`` repeats them over
  environments p = (q, theta_v, m), all grids in one ensemble;
* ``chi``: the root-mean-square gauge-depth misfit over experiments and gauges
  (Eq. eq_chi_6experim);
* ``chi_surfaces``: chi over the grid for the experiment subsets (cases I-IV) of Sec. 4.3;
* ``hooke_jeeves``: Hooke and Jeeves' pattern search (exploratory moves coordinate by
  coordinate, pattern moves, step halving).  Each exploratory move evaluates the 3 x 3
  stencil around its base point in one batch, which holds every point the sequential
  move can visit in two dimensions, so the search takes exactly the sequential
  algorithm's decisions while the solver runs batched.

Only host logic and argument marshalling live here; every solver step runs in the
ensemble kernel.  The paper's flume measurements are not available: ``synthetic_gauges``
makes the "measured" depths with the solver itself at known coefficients, and the
estimation then has to recover them.
"""
from __future__ import annotations

import itertools
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs
from .ensemble import Ensemble

LAMBDA = ((0.0025, 0.0185), (55.0, 80.0))      # the search box of Sec. 4.3 (alpha_s, alpha_p)
GRID = (21, 26)                                   # its regular grid


@dataclass
class FlumeStudy:
    """Discretisation and run length shared by every flume run of a study."""
    l: float = 0.1
    t_end: float = 600.0
    tailwater: float = 0.1
    n_gauges: int = 17
    experiments: tuple = inputs.FLUME["q"]        # (layout, q_l [m^3/s]) pairs
    tuning: tuple | None = None                   # ensemble launch shape (None: autotune)
    runs: int = 0                                 # scenarios run so far
    cell_updates: int = 0                         # cells x time steps of those runs
    seconds: float = 0.0                          # wall time, end to end (build, tune, solve, read back)
    solve_seconds: float = 0.0                    # wall time of the ensemble launches alone
    tune_seconds: float = 0.0                     # wall time of the launch-shape search

    def scenario(self, alpha_s: float, alpha_p: float, layout: int, q_l: float, theta_v: float | None = None,
                 slope: float | None = None):
        sc = inputs.flume(q_l, layout, alpha_s, alpha_p, l=self.l, tailwater=self.tailwater, t_end=self.t_end,
                          theta_v=theta_v, slope=slope)
        sc.viscosity = True
        return sc


def steady_depths(study: FlumeStudy, scenarios: list) -> list[np.ndarray]:
    """Runs the scenarios to their end time in one ensemble and returns each depth field
    (rows x cols)."""
    t0 = time.perf_counter()
    E = Ensemble(scenarios)
    try:
        tuning = study.tuning
        t1 = time.perf_counter()
        if tuning is None:
            study.tuning = tuning = E.autotune(max_steps=200).as_tuple()
        t2 = time.perf_counter()
        E.run(tuning)                     # returns once the launch has finished
        t3 = time.perf_counter()
        out = []
        for s, sc in enumerate(scenarios):
            t, steps = E.clock(s)
            if t < sc.t_end * (1.0 - 1e-12):
                raise RuntimeError(f"scenario {s} stopped at t = {t} before {sc.t_end}")
            study.cell_updates += steps * sc.n
            out.append(E.fields(s)[0])
    finally:
        E.close()
    study.runs += len(scenarios)
    study.tune_seconds += t2 - t1
    study.solve_seconds += t3 - t2
    study.seconds += time.perf_counter() - t0
    return out


def h_bar(h: np.ndarray, sc) -> float:
    """Mean depth over the cells whose centre lies at x >= 9 m (Eq. eq_h_bar)."""
    x, _ = inputs.cell_centres(sc.rows, sc.cols, sc.l)
    return float(np.asarray(h, np.float64)[x >= 9.0].mean())


def gauge_depths(h: np.ndarray, sc, n: int) -> np.ndarray:
    return np.asarray(h, np.float64).ravel()[inputs.flume_gauges(sc, n)]


def sensitivity(H: np.ndarray, d_s: float, d_p: float) -> tuple[float, float]:
    """delta_s and delta_p of Sec. 4.3 from h_bar on the grid H[i, j] = h_bar(alpha_s^i,
    alpha_p^j): the forward differences along each axis divided by the grid step, averaged
    over the (N_s - 1) N_p, respectively N_s (N_p - 1), pairs."""
    H = np.asarray(H, np.float64)
    return float((np.diff(H, axis=0) / d_s).mean()), float((np.diff(H, axis=1) / d_p).mean())


def grid_points(ns: int = GRID[0], np_: int = GRID[1], box=LAMBDA):
    """The regular grid alpha_s^i = lo_s + (i - 1) d_s, alpha_p^j = lo_p + (j - 1) d_p."""
    (s0, s1), (p0, p1) = box
    return np.linspace(s0, s1, ns), np.linspace(p0, p1, np_)


def sensitivity_grid(study: FlumeStudy, layout: int = 1, q_l: float = 0.015, ns: int = GRID[0],
                     np_: int = GRID[1], box=LAMBDA) -> dict:
    """h_bar over the (alpha_s, alpha_p) grid of one experiment, all grid points in one
    ensemble, and the two sensitivities."""
    a_s, a_p = grid_points(ns, np_, box)
    scs = [study.scenario(s, p, layout, q_l) for s in a_s for p in a_p]
    hs = steady_depths(study, scs)
    H = np.array([h_bar(h, sc) for h, sc in zip(hs, scs)]).reshape(ns, np_)
    ds, dp = sensitivity(H, a_s[1] - a_s[0], a_p[1] - a_p[0])
    return dict(alpha_s=a_s, alpha_p=a_p, h_bar=H, delta_s=ds, delta_p=dp)


def sensitivity_sweep(study: FlumeStudy, envs: list, layout: int = 1, ns: int = GRID[0], np_: int = GRID[1],
                      box=LAMBDA) -> list[dict]:
    """delta_s and delta_p as functions of the environment p = (q, theta_v, m) (Sec. 4.3):
    one (alpha_s, alpha_p) grid per environment dict(q=..., theta_v=..., slope=...), every
    grid of every environment in one ensemble."""
    a_s, a_p = grid_points(ns, np_, box)
    scs = [study.scenario(s, p, layout, e["q"], e.get("theta_v"), e.get("slope")) for e in envs for s in a_s
           for p in a_p]
    hs = steady_depths(study, scs)
    Hb = np.array([h_bar(h, sc) for h, sc in zip(hs, scs)]).reshape(len(envs), ns, np_)
    out = []
    for e, H in zip(envs, Hb):
        ds, dp = sensitivity(H, a_s[1] - a_s[0], a_p[1] - a_p[0])
        out.append(dict(env=dict(e), h_bar=H, delta_s=ds, delta_p=dp))
    return out


def chi(h_exp: np.ndarray, h_sim: np.ndarray) -> float:
    """Root-mean-square misfit over every experiment and gauge (Eq. eq_chi_6experim)."""
    d = np.asarray(h_exp, np.float64) - np.asarray(h_sim, np.float64)
    return float(np.sqrt(np.mean(d * d)))


def simulate_gauges(study: FlumeStudy, points: list) -> np.ndarray:
    """Gauge depths [len(points), experiments, gauges] for each (alpha_s, alpha_p) point,
    every point and experiment in one ensemble."""
    scs = [study.scenario(s, p, lay, q) for (s, p) in points for (lay, q) in study.experiments]
    hs = steady_depths(study, scs)
    g = np.array([gauge_depths(h, sc, study.n_gauges) for h, sc in zip(hs, scs)])
    return g.reshape(len(points), len(study.experiments), study.n_gauges)


def synthetic_gauges(study: FlumeStudy, alpha_s: float, alpha_p: float) -> np.ndarray:
    """Stand-in for the flume measurements: the solver's own gauge depths at known
    coefficients, [experiments, gauges]."""
    return simulate_gauges(study, [(alpha_s, alpha_p)])[0]


# The experiment subsets of Sec. 4.3, as indices into inputs.FLUME["q"]: one experiment
# (layout 1, 15 l/s), the three of layout 1, the three of layout 2, all six.
CASES = {"I": (1,), "II": (0, 1, 2), "III": (3, 4, 5), "IV": (0, 1, 2, 3, 4, 5)}


def chi_surfaces(study: FlumeStudy, h_exp: np.ndarray, ns: int = GRID[0], np_: int = GRID[1], box=LAMBDA,
                 cases=CASES) -> dict:
    """chi over the (alpha_s, alpha_p) grid for each case of Sec. 4.3: every grid point and
    experiment in one ensemble, each case's surface from its subset of experiments.
    h_exp: [experiments, gauges] for study.experiments."""
    a_s, a_p = grid_points(ns, np_, box)
    g = simulate_gauges(study, [(s, p) for s in a_s for p in a_p])          # [points, experiments, gauges]
    out = {}
    for name, idx in cases.items():
        idx = list(idx)
        chi_grid = np.array([chi(h_exp[idx], gi[idx]) for gi in g]).reshape(ns, np_)
        i, j = np.unravel_index(np.argmin(chi_grid), chi_grid.shape)
        out[name] = dict(chi=chi_grid, argmin=(float(a_s[i]), float(a_p[j])), min=float(chi_grid[i, j]))
    return dict(alpha_s=a_s, alpha_p=a_p, cases=out)


@dataclass
class Search:
    x: np.ndarray                 # minimiser found (in the caller's coordinates)
    f: float
    evals: int                    # distinct points evaluated
    batches: int                  # batched evaluations
    path: list = field(default_factory=list)   # accepted base points


def hooke_jeeves(f_batch, x0, step, lo, hi, shrink: float = 0.5, tol: float = 1e-3, max_batches: int = 500) -> Search:
    """Minimises f over the box [lo, hi] by Hooke and Jeeves' pattern search in the
    coordinates u = (x - lo) / (hi - lo) (a point outside the box counts as +inf).

    f_batch(list of points) -> values.  From a base point b the exploratory move tries, in
    each coordinate in turn, +step then -step, keeping a trial when it lowers f; if the
    move ends below f(b), the pattern point x + (x - b) becomes the next centre of
    exploration while it keeps improving; otherwise the step shrinks, until it is below
    tol.  The exploratory move's points all lie on the 3 x 3 stencil around its centre
    (two coordinates), which is evaluated in one batch."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    span = hi - lo
    d = len(lo)
    cache: dict = {}
    counts = [0, 0]

    def key(u):
        return tuple(np.round(u, 12))

    def evaluate(us):
        todo = []
        for u in us:
            k = key(u)
            if k in cache:
                continue
            if np.any(u < -1e-12) or np.any(u > 1.0 + 1e-12):
                cache[k] = np.inf
            else:
                todo.append(k)
                cache[k] = None
        todo = list(dict.fromkeys(todo))
        if todo:
            vals = f_batch([lo + np.array(k) * span for k in todo])
            counts[0] += len(todo)
            counts[1] += 1
            for k, v in zip(todo, vals):
                cache[k] = float(v)
        return [cache[key(u)] for u in us]

    def explore(c, fc, s):
        offsets = [np.array(o, np.float64) for o in itertools.product((-1.0, 0.0, 1.0), repeat=d)]
        evaluate([c + o * s for o in offsets])
        x, fx = c.copy(), fc
        for i in range(d):
            for sg in (1.0, -1.0):
                t = x.copy()
                t[i] += sg * s[i]
                ft = evaluate([t])[0]
                if ft < fx:
                    x, fx = t, ft
                    break
        return x, fx

    s = np.asarray(step, np.float64) / span
    b = (np.asarray(x0, np.float64) - lo) / span
    fb = evaluate([b])[0]
    path = [lo + b * span]
    while np.max(s) >= tol and counts[1] < max_batches:
        x, fx = explore(b, fb, s)
        if fx < fb:
            while True:
                prev, b, fb = b, x, fx
                path.append(lo + b * span)
                p = b + (b - prev)
                fp = evaluate([p])[0]
                x, fx = explore(p, fp, s)
                if not fx < fb:
                    break
        else:
            s = s * shrink
    return Search(x=lo + b * span, f=fb, evals=counts[0], batches=counts[1], path=path)


def calibrate(study: FlumeStudy, h_exp: np.ndarray, x0=None, step=None, tol: float = 1e-3, box=LAMBDA) -> Search:
    """Estimates (alpha_s, alpha_p) by minimising chi against the gauge depths h_exp
    [experiments, gauges] with the pattern search, each batch of trial points solved in
    one ensemble."""
    lo = np.array([box[0][0], box[1][0]])
    hi = np.array([box[0][1], box[1][1]])
    x0 = (lo + hi) / 2 if x0 is None else np.asarray(x0, np.float64)
    step = (hi - lo) / 4 if step is None else np.asarray(step, np.float64)

    def f_batch(points):
        g = simulate_gauges(study, [tuple(p) for p in points])
        return [chi(h_exp, gi) for gi in g]

    return hooke_jeeves(f_batch, x0, step, lo, hi, tol=tol)
