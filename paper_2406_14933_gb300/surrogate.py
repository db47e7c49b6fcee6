"""The learned hydrograph surrogate (not in the paper; this library's addition).

A small MLP stands in for whole hillslope runs: from a scenario's slope, vegetation cover,
porosity, plant drag and its hyetograph it predicts the outlet hydrograph.  It is trained
on hydrographs the solver itself produces (the hillslope ensemble of Sec. 2 scenarios run
to 6400 s), and the solver remains the reference: at serving time a sample of the queries is
re-solved, their error measured, and the solver's hydrograph replaces the surrogate's
wherever the relative L2 error exceeds the tolerance.

Orchestration and argument marshalling only.  The solver runs are ``asx_ensemble_run``
(the persistent ensemble kernel), the network's forward, backward and Adam steps are the
``asx_mlp_*`` tensor-core kernels, and the error check with fallback is
``asx_surrogate_check``.  PyTorch holds device buffers and does the minibatch gathers.

Encoding (Sec. 2 quantities, normalised):
* inputs (36): slope, cover fraction, porosity theta of vegetated cells and plant drag
  alpha_p, each mapped linearly from the generator's range onto [-1, 1]; then the
  hyetograph as 32 bin means of the rain rate r(t) over 0-3600 s (bins of 112.5 s), in
  units of 150 mm/h.  The mean is the exact integral of the piecewise-linear rain table
  (zero outside its first and last time) over the bin.
* outputs (128): the outlet discharge averaged over the 128 intervals of 50 s in 0-6400 s
  (the solver's hydrograph), divided by the scenario's peak rain inflow A * max r(t),
  A = rows * cols * sigma the raster's area.  The relative L2 error of a hydrograph is the
  same in either unit.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import asx as _a
from .inputs import MM_PER_H, Scenario, constant_rain, ensemble_member, member_params

N_IN, N_HYDRO_OUT, N_PARAMS = _a.ASX_MLP_IN, _a.ASX_MLP_OUT, _a.ASX_MLP_PARAMS
N_HYETO, HYETO_T = 32, 3600.0
HYDRO_DT = 50.0
HYDRO_T = HYDRO_DT * N_HYDRO_OUT            # 6400 s
R_REF = 150.0 * MM_PER_H                    # rain-rate unit of the hyetograph inputs [m/s]
RANGES = (("slope", 0.02, 0.30), ("cover", 0.0, 0.80), ("theta", 0.70, 0.95), ("alpha_p", 20.0, 100.0))
LAYERS = ((256, 36), (256, 256), (256, 256), (128, 256))   # (out, in) of W1..W4

TRAIN_SEED0 = 5_000_000        # training scenario i draws seed TRAIN_SEED0 + i
HELD_OUT_SEED0 = 5_500_000     # held-out scenarios: a disjoint seed range
QUERY_SEED0 = 6_000_000        # serving queries


# ----------------------------------------------------------------------------- encoding

def cumulative_rain(rain_t, rain_r, t) -> np.ndarray:
    """Integral of the piecewise-linear rain rate from 0 to each t [m]."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    rt = np.asarray(rain_t, dtype=np.float64)
    rr = np.asarray(rain_r, dtype=np.float64)
    for k in range(rt.size - 1):
        t0, t1, r0, r1 = rt[k], rt[k + 1], rr[k], rr[k + 1]
        if not t1 > t0:
            continue
        u = np.clip(t, t0, t1) - t0
        out += r0 * u + (r1 - r0) * u * u / (2.0 * (t1 - t0))
    return out


def hyetograph(rain_t, rain_r, n: int = N_HYETO, t_end: float = HYETO_T) -> np.ndarray:
    """Mean rain rate over n equal bins of [0, t_end] [m/s]."""
    edges = np.linspace(0.0, t_end, n + 1)
    return np.diff(cumulative_rain(rain_t, rain_r, edges)) / (t_end / n)


def encode(meta: dict, rain_t, rain_r) -> np.ndarray:
    """The 36 network inputs from a member's scalars and its rain table (float32)."""
    out = np.empty(N_IN, dtype=np.float32)
    for i, (key, lo, hi) in enumerate(RANGES):
        out[i] = 2.0 * (float(meta[key]) - lo) / (hi - lo) - 1.0
    out[len(RANGES):] = hyetograph(rain_t, rain_r) / R_REF
    return out


def features(sc: Scenario) -> np.ndarray:
    """The 36 network inputs of a hillslope-ensemble scenario (float32)."""
    return encode(sc.meta, sc.rain_t, sc.rain_r)


def query_features(seed0: int, count: int, n: int = 256, l: float = 2.0, start: int = 0):
    """Features (count x 36) and output scales of members start .. start+count-1, from
    their scalar draws alone (no fields are built)."""
    X = np.empty((count, N_IN), dtype=np.float32)
    S = np.empty(count, dtype=np.float64)
    sigma = 1.5 * math.sqrt(3.0) * l * l
    for i in range(count):
        d = member_params(start + i, base_seed=seed0, n_override=n)
        rt, rr = constant_rain(d["rain_mm_h"], d["rain_s"])
        X[i] = encode(d, rt, rr)
        S[i] = n * n * sigma * float(np.max(rr))
    return X, S


def discharge_scale(sc: Scenario) -> float:
    """A * max r(t) [m^3/s]: the unit of the network's outputs."""
    sigma = 1.5 * math.sqrt(3.0) * sc.l * sc.l
    return float(sc.rows * sc.cols * sigma * max(float(np.max(sc.rain_r)), 1e-30))


COVER_CORR_M = 16.0            # correlation length of the vegetation-cover field [m]


def scenario(seed0: int, i: int, n: int = 256, l: float = 2.0) -> Scenario:
    """Member i of a hillslope ensemble at n x n cells of edge l (cover patches of a fixed
    physical size, COVER_CORR_M), run to 6400 s with the hydrograph sampled every 50 s."""
    sc = ensemble_member(i, base_seed=seed0, n_override=n, l=l, t_end=HYDRO_T, corr_cells=COVER_CORR_M / l)
    sc.sample_dt = HYDRO_DT
    return sc


def _make(args):
    seed0, i, n, l = args
    sc = scenario(seed0, i, n, l)
    return sc, features(sc), discharge_scale(sc)


def make_scenarios(seed0: int, count: int, n: int = 256, l: float = 2.0, workers: int = 0, start: int = 0):
    """Scenarios start .. start+count-1 with their features (count x 36) and output scales.
    workers > 1 generates them in a pool of spawned processes."""
    jobs = [(seed0, start + i, n, l) for i in range(count)]
    if workers and workers > 1 and count >= 4 * workers:
        # spawned workers re-import the caller's main module, which must therefore be a
        # file guarded by `if __name__ == "__main__"`; a broken pool raises, it never hangs
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
            res = list(pool.map(_make, jobs, chunksize=max(1, count // (8 * workers))))
    else:
        res = [_make(j) for j in jobs]
    scs = [r[0] for r in res]
    X = np.stack([r[1] for r in res]) if res else np.zeros((0, N_IN), np.float32)
    S = np.array([r[2] for r in res], dtype=np.float64)
    return scs, X, S


# ----------------------------------------------------------------------------- the solver side

@dataclass
class SolveStats:
    scenarios: int = 0
    seconds: float = 0.0            # wall time of the ensemble runs (device work, synchronised)
    wall: float = 0.0               # the same plus upload of the fields and readback
    cell_updates: float = 0.0

    @property
    def hydrographs_per_s(self) -> float:
        """Solved hydrographs per second of wall time, uploads and readback included."""
        return self.scenarios / self.wall if self.wall > 0 else 0.0


def solve(scs: list[Scenario], scales: np.ndarray, chunk: int = 2048, tuning=None,
          stats: SolveStats | None = None) -> np.ndarray:
    """Runs every scenario on the GPU (the persistent ensemble kernel, `chunk` scenarios per
    launch) and returns their hydrographs in output units (len x 128, float32)."""
    import torch

    from .ensemble import Ensemble
    Y = np.zeros((len(scs), N_HYDRO_OUT), dtype=np.float32)
    for c0 in range(0, len(scs), chunk):
        part = scs[c0:c0 + chunk]
        tw = time.perf_counter()
        ens = Ensemble(part, n_samples=N_HYDRO_OUT)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ens.run(tuning)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            for j in range(len(part)):
                q = ens.hydrograph(j, N_HYDRO_OUT)
                if q.size != N_HYDRO_OUT:
                    raise RuntimeError(f"scenario {c0 + j}: {q.size} hydrograph samples, expected {N_HYDRO_OUT}")
                Y[c0 + j] = q / scales[c0 + j]
            if stats is not None:
                stats.scenarios += len(part)
                stats.seconds += dt
                stats.wall += time.perf_counter() - tw
                stats.cell_updates += float(sum(ens.clock(j)[1] * sc.rows * sc.cols for j, sc in enumerate(part)))
        finally:
            ens.close()
    return Y


def dataset(seed0: int, count: int, n: int = 256, l: float = 2.0, workers: int = 0, chunk: int = 2048,
            stats: SolveStats | None = None, tuning=None):
    """Features (count x 36) and solver hydrographs (count x 128, output units) of members
    0 .. count-1, generated and solved `chunk` at a time so that host memory stays bounded."""
    X = np.empty((count, N_IN), dtype=np.float32)
    Y = np.empty((count, N_HYDRO_OUT), dtype=np.float32)
    for c0 in range(0, count, chunk):
        k = min(chunk, count - c0)
        scs, X[c0:c0 + k], sc_scale = make_scenarios(seed0, k, n, l, workers, start=c0)
        Y[c0:c0 + k] = solve(scs, sc_scale, chunk=chunk, tuning=tuning, stats=stats)
        del scs
    return X, Y


def autotune(n: int = 256, l: float = 2.0, count: int = 152, max_steps: int = 50):
    """Ensemble tuning for members of this size (the library's autotuner)."""
    from .ensemble import Ensemble
    scs, _, _ = make_scenarios(TRAIN_SEED0, count, n, l)
    ens = Ensemble(scs, n_samples=N_HYDRO_OUT)
    try:
        return ens.autotune(max_steps)
    finally:
        ens.close()


# ----------------------------------------------------------------------------- the network

def init_params(rng: np.random.Generator) -> np.ndarray:
    """He-normal weights, zero biases, in the packed layout (W1, b1, ..., W4, b4)."""
    parts = []
    for o, i in LAYERS:
        parts.append(rng.standard_normal(o * i) * math.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == N_PARAMS
    return p


def rel_l2(y, ref) -> np.ndarray:
    """Per-row relative L2 error ||y - ref|| / ||ref||."""
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.linalg.norm(y - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-30)


@dataclass
class ServeReport:
    queries: int
    checked: int
    replaced: int
    rel_err: np.ndarray                     # per checked query, before fallback
    infer_seconds: float                    # the network's forward pass over every query
    check_seconds: float                    # re-solving the sample plus the check kernel
    solver: SolveStats = field(default_factory=SolveStats)

    @property
    def hydrographs_per_s(self) -> float:
        """Served hydrographs per second, the sampled solver check included."""
        return self.queries / (self.infer_seconds + self.check_seconds)


class Surrogate:
    """The MLP on one device; `fit` trains it on device tensors with Adam."""

    def __init__(self, device: int = 0, max_batch: int = 65536, seed: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.max_batch = int(max_batch)
        self.handle = _a.asx_mlp_create(device, None, self.max_batch)
        self.set_params(init_params(np.random.default_rng(seed)))

    def set_params(self, p: np.ndarray):
        _a.asx_mlp_set_params(self.handle, np.ascontiguousarray(p, dtype=np.float32))

    def params(self) -> np.ndarray:
        out = np.empty(N_PARAMS, np.float32)
        _a.asx_mlp_get_params(self.handle, out)
        return out

    def _dev(self, a):
        t = self.torch
        if isinstance(a, t.Tensor):
            return a.to(self.device, t.float32).contiguous()
        return t.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=self.device)

    def fit(self, X, Y, epochs: int, batch: int = 512, lr: float = 1e-3, lr_final: float = 1e-5,
            weight_decay: float = 0.0, seed: int = 0, log_every: int = 0) -> dict:
        """Adam over `epochs` passes of the data in shuffled minibatches, the learning rate
        decaying from lr to lr_final on a cosine.  Returns the training history and time."""
        t = self.torch
        X, Y = self._dev(X), self._dev(Y)
        n = X.shape[0]
        batch = min(batch, n, self.max_batch)
        steps_per_epoch = n // batch
        total = epochs * steps_per_epoch
        gen = t.Generator(device=self.device)
        gen.manual_seed(seed)
        hist = []
        t.cuda.synchronize()
        t0 = time.perf_counter()
        step = 0
        for ep in range(epochs):
            perm = t.randperm(n, device=self.device, generator=gen)
            Xp, Yp = X[perm], Y[perm]
            for b in range(steps_per_epoch):
                frac = step / max(total - 1, 1)
                lr_s = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * frac))
                last = b == steps_per_epoch - 1 and log_every and (ep + 1) % log_every == 0
                loss = _a.asx_mlp_train_step(self.handle, batch, Xp[b * batch:(b + 1) * batch].data_ptr(),
                                             Yp[b * batch:(b + 1) * batch].data_ptr(), lr_s, weight_decay,
                                             _a.ASX_PTR_DEVICE, want_loss=bool(last))
                if last:
                    hist.append((ep + 1, loss))
                step += 1
        t.cuda.synchronize()
        secs = time.perf_counter() - t0
        return dict(epochs=epochs, steps=step, seconds=secs, epochs_per_s=epochs / secs if secs > 0 else 0.0,
                    history=hist)

    def predict(self, X):
        """Forward pass over every row of X; returns a (n, 128) float32 CUDA tensor."""
        t = self.torch
        X = self._dev(X)
        Y = t.empty((X.shape[0], N_HYDRO_OUT), dtype=t.float32, device=self.device)
        if X.shape[0]:
            _a.asx_mlp_forward(self.handle, X.shape[0], X.data_ptr(), Y.data_ptr(), _a.ASX_PTR_DEVICE)
        return Y

    def check(self, Y, idx, ref, tol: float = 0.05):
        """asx_surrogate_check: measures the rows idx of Y against the solver's `ref` and
        replaces those whose relative L2 error exceeds tol.  Returns (rel_err, replaced)."""
        t = self.torch
        idx_d = t.as_tensor(np.asarray(idx, dtype=np.int32), device=self.device)
        ref_d = self._dev(ref)
        err = t.empty(idx_d.numel(), dtype=t.float32, device=self.device)
        nrep = t.zeros(1, dtype=t.int32, device=self.device)
        _a.asx_surrogate_check(Y.shape[0], idx_d.numel(), idx_d.data_ptr(), Y.data_ptr(), ref_d.data_ptr(), tol,
                               err.data_ptr(), nrep.data_ptr(), t.cuda.current_stream(self.device).cuda_stream)
        return err.cpu().numpy(), int(nrep.item())

    def serve(self, X, scales: np.ndarray, scenarios_of, frac: float = 0.01, tol: float = 0.05,
              seed: int = 0, chunk: int = 2048, tuning=None):
        """Inference over every query, then the solver check of a random `frac` of them
        (at least one) with fallback.  scales[i] is query i's output unit and
        scenarios_of(idx) builds the full scenarios of the sampled queries (host input
        synthesis, not timed).  Returns (Y on the device, ServeReport)."""
        t = self.torch
        Xd = self._dev(X)
        n = Xd.shape[0]
        t.cuda.synchronize()
        t0 = time.perf_counter()
        Y = self.predict(Xd)
        t.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        k = min(n, max(1, int(math.ceil(frac * n))))
        idx = np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))
        scs = scenarios_of(idx)
        st = SolveStats()
        t1 = time.perf_counter()
        ref = solve(scs, np.asarray(scales)[idx], chunk=chunk, tuning=tuning, stats=st)
        err, nrep = self.check(Y, idx, ref, tol)
        t.cuda.synchronize()
        t_chk = time.perf_counter() - t1
        return Y, ServeReport(n, k, nrep, err, t_inf, t_chk, st)

    def close(self):
        if getattr(self, "handle", None):
            _a.asx_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- the whole pipeline

def pipeline(n: int = 256, l: float = 2.0, n_train: int = 20000, n_held: int = 1000, n_queries: int = 65536,
             epochs: int = 150, batch: int = 256, lr: float = 1e-3, frac: float = 0.01, tol: float = 0.05,
             workers: int = 0, chunk: int = 2048, seed: int = 0, log=None) -> tuple[dict, "Surrogate"]:
    """Generate training and held-out runs with the solver, train, evaluate on the held-out
    runs, then serve n_queries queries with the solver check.  Returns (report, model)."""
    import torch
    say = log or (lambda *_: None)
    tuning = autotune(n, l)
    say(f"autotuned: cluster {tuning.cluster} threads {tuning.threads} cells/thread {tuning.cells_per_thread} "
        f"tile rows {tuning.tile_rows} split {tuning.split}")
    st_train = SolveStats()
    X, Y = dataset(TRAIN_SEED0, n_train, n, l, workers, chunk, st_train, tuning)
    say(f"training runs: {n_train} in {st_train.wall:.1f} s ({st_train.hydrographs_per_s:.1f} hydrographs/s)")
    Xh, Yh = dataset(HELD_OUT_SEED0, n_held, n, l, workers, chunk, None, tuning)
    model = Surrogate(max_batch=max(n_queries, batch), seed=seed)
    fit = model.fit(X, Y, epochs=epochs, batch=batch, lr=lr, seed=seed, log_every=max(1, epochs // 5))
    say(f"trained: {epochs} epochs in {fit['seconds']:.1f} s, loss {fit['history']}")
    P = model.predict(Xh).cpu().numpy()
    e = rel_l2(P, Yh)
    mean_h = Y.mean(axis=0, keepdims=True)
    e_mean = rel_l2(np.repeat(mean_h, len(Yh), axis=0), Yh)
    held = dict(count=n_held, mean=float(e.mean()), median=float(np.median(e)), p90=float(np.quantile(e, 0.9)),
                max=float(e.max()), aggregate=float(np.linalg.norm(P - Yh) / np.linalg.norm(Yh)),
                frac_within_tol=float(np.mean(e <= tol)), mean_hydrograph_baseline=float(e_mean.mean()))
    say(f"held-out rel L2: {held}")
    Xq, Sq = query_features(QUERY_SEED0, n_queries, n, l)

    def scenarios_of(idx):
        return [scenario(QUERY_SEED0, int(i), n, l) for i in idx]

    # one untimed pass so that the timed inference sees warm kernels
    model.predict(torch.as_tensor(Xq[:min(len(Xq), 1024)], device=model.device))
    _, rep = model.serve(Xq, Sq, scenarios_of, frac=frac, tol=tol, seed=seed + 1, chunk=chunk, tuning=tuning)
    ok = rep.rel_err[np.isfinite(rep.rel_err)]
    # the checked sample estimates the share of unchecked served hydrographs within tol
    # (binomial standard error beside it); checked ones are within tol after the fallback
    p_in = float(np.mean(ok <= tol)) if ok.size else None
    se = float(np.sqrt(p_in * (1 - p_in) / ok.size)) if ok.size else None
    cf = rep.checked / max(rep.queries, 1)
    serve = dict(queries=rep.queries, checked=rep.checked, replaced=rep.replaced,
                 checked_mean_rel_l2=float(ok.mean()) if ok.size else None,
                 checked_p90_rel_l2=float(np.quantile(ok, 0.9)) if ok.size else None,
                 checked_frac_within_tol=p_in, checked_frac_within_tol_stderr=se,
                 served_frac_within_tol_estimate=(cf + (1 - cf) * p_in) if ok.size else None,
                 infer_seconds=rep.infer_seconds, queries_per_s=rep.queries / rep.infer_seconds,
                 check_seconds=rep.check_seconds, served_hydrographs_per_s=rep.hydrographs_per_s,
                 solver_hydrographs_per_s=rep.solver.hydrographs_per_s,
                 gain=rep.hydrographs_per_s / rep.solver.hydrographs_per_s if rep.solver.wall > 0 else None)
    say(f"served: {serve}")
    report = dict(workload=f"hillslope ensemble members {n}x{n}, l={l} m, 6400 s", n=n, l=l,
                  train=dict(runs=n_train, solver_wall_s=st_train.wall, solver_hydrographs_per_s=st_train.hydrographs_per_s,
                             solver_cell_updates_per_s=st_train.cell_updates / st_train.seconds if st_train.seconds else 0.0,
                             epochs=epochs, batch=batch, steps=fit["steps"], fit_seconds=fit["seconds"],
                             epochs_per_s=fit["epochs_per_s"],
                             final_loss=fit["history"][-1][1] if fit["history"] else None),
                  held_out=held, serve=serve,
                  tuning=dict(cluster=tuning.cluster, threads=tuning.threads, cells_per_thread=tuning.cells_per_thread,
                              tile_rows=tuning.tile_rows, split=tuning.split))
    return report, model


def main(argv=None):
    import argparse
    import json
    import os
    ap = argparse.ArgumentParser(description="Train the hydrograph surrogate on solver runs and serve queries.")
    ap.add_argument("--n", type=int, default=256, help="raster side [cells]")
    ap.add_argument("--l", type=float, default=2.0, help="hexagon edge [m]")
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--held-out", type=int, default=1000)
    ap.add_argument("--queries", type=int, default=65536)
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--out", default=None, help="directory for report.json and params.npy")
    a = ap.parse_args(argv)
    rep, model = pipeline(a.n, a.l, a.train, a.held_out, a.queries, a.epochs, workers=a.workers,
                          log=lambda m: print(m, flush=True))
    print(json.dumps(rep))
    if a.out:
        os.makedirs(a.out, exist_ok=True)
        with open(os.path.join(a.out, "report.json"), "w") as f:
            json.dump(rep, f, indent=1)
        np.save(os.path.join(a.out, "params.npy"), model.params())
    model.close()


if __name__ == "__main__":
    main()
