"""Convenience wrapper: an ``asx_ensemble`` built from a list of ``inputs.Scenario``.

Argument marshalling only; every scenario is advanced on the GPU by the persistent
ensemble kernel of libasx.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import asx as _a
from .inputs import Scenario


def _f32(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(shape))


def _uniform(arr):
    a = np.asarray(arr).reshape(-1)
    if not np.all(a == a[0]):
        raise ValueError("ensemble scenarios take scalar alpha_s / alpha_p")
    return float(a[0])


class Ensemble:
    def __init__(self, scenarios: list[Scenario], n_samples: int | None = None, device: int = 0,
                 stream: int | None = None, max_steps: int = 0):
        self.scenarios = scenarios
        self._keep = []
        descs = []
        for sc in scenarios:
            d = _a.asx_scenario_desc()
            d.rows, d.cols, d.edge_m = sc.rows, sc.cols, sc.l
            for s in range(4):
                d.bc[s] = int(sc.bc[s])
                d.free_begin[s], d.free_end[s] = (int(v) for v in sc.free_range[s])
            d.g, d.cfl, d.dt_max = sc.g, sc.cfl, sc.dt_max
            d.alpha_s, d.alpha_p = _uniform(sc.alpha_s), _uniform(sc.alpha_p)
            rt = np.ascontiguousarray(sc.rain_t, dtype=np.float64)
            rr = np.ascontiguousarray(sc.rain_r, dtype=np.float64)
            self._keep += [rt, rr]
            dp = C.POINTER(C.c_double)
            d.n_rain = int(rt.size)
            d.rain_t, d.rain_r = rt.ctypes.data_as(dp), rr.ctypes.data_as(dp)
            d.t_end = sc.t_end
            d.sample_dt = sc.sample_dt
            if n_samples is not None:
                d.max_samples = int(n_samples)
            else:
                d.max_samples = int(np.ceil(sc.t_end / sc.sample_dt)) + 2 if sc.sample_dt > 0 else 0
            d.max_steps = int(max_steps)
            for s in range(4):
                d.bc_q[s], d.bc_h[s], d.bc_u[s] = float(sc.bc_q[s]), float(sc.bc_h[s]), float(sc.bc_u[s])
            d.viscosity = int(bool(sc.viscosity))
            d.tau, d.h_dry = float(sc.tau), float(sc.h_dry)
            descs.append(d)
        self.handle = _a.asx_create_ensemble(descs, stream, device)
        for i, sc in enumerate(scenarios):
            sh = (sc.rows, sc.cols)
            _a.asx_ensemble_set_fields(self.handle, i, np.ascontiguousarray(np.asarray(sc.z, np.float64).reshape(sh)),
                                       _f32(sc.theta, sh), _f32(sc.h0, sh),
                                       _f32(sc.v1_0, sh), _f32(sc.v2_0, sh), _a.ASX_PTR_HOST)

    def autotune(self, max_steps=50):
        return _a.asx_ensemble_autotune(self.handle, max_steps)

    def run(self, tuning=None):
        if tuning is not None and not isinstance(tuning, _a.asx_ensemble_tuning):
            tuning = _a.asx_ensemble_tuning(*tuning)
        _a.asx_ensemble_run(self.handle, tuning)

    def ledger(self, s):
        return _a.asx_ensemble_ledger(self.handle, s)

    def clock(self, s):
        return _a.asx_ensemble_get_clock(self.handle, s)

    def state(self, s):
        sc = self.scenarios[s]
        sh = (sc.rows, sc.cols)
        mh, ml, v1, v2 = (np.empty(sh, np.float32) for _ in range(4))
        _a.asx_ensemble_get_state(self.handle, s, mh, ml, v1, v2, _a.ASX_PTR_HOST)
        return mh, ml, v1, v2

    def fields(self, s):
        sc = self.scenarios[s]
        sh = (sc.rows, sc.cols)
        h, v1, v2 = (np.empty(sh, np.float32) for _ in range(3))
        _a.asx_ensemble_get_fields(self.handle, s, h, v1, v2, _a.ASX_PTR_HOST)
        return h, v1, v2

    def hydrograph(self, s, cap=1 << 20):
        return _a.asx_ensemble_get_hydrograph(self.handle, s, cap)[0]

    def close(self):
        if self.handle:
            _a.asx_destroy_ensemble(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
