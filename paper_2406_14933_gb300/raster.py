"""Convenience wrapper: one ``asx_raster`` handle built from an ``inputs.Scenario``.

Only argument marshalling: builds the C descriptor / parameter structs, copies numpy
fields in through ``asx_set_fields`` and reads results back.  All work runs in libasx.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import asx as _a
from .inputs import Scenario


def _f32(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(shape))


def _f64(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


def _uniform(arr, what):
    a = np.asarray(arr).reshape(-1)
    if a.size and not np.all(a == a[0]):
        raise ValueError(f"{what} must be uniform unless land-cover classes are used")
    return float(a[0]) if a.size else 0.0


class Raster:
    def __init__(self, sc: Scenario, device: int = 0, stream: int | None = None,
                 max_samples: int | None = None, use_classes: bool | None = None, fp64: bool = False):
        self.sc = sc
        use_classes = (sc.cls is not None) if use_classes is None else use_classes
        nc = int(len(sc.class_theta)) if use_classes else 0
        if max_samples is None:
            max_samples = int(np.ceil(sc.t_end / sc.sample_dt)) + 2 if sc.sample_dt > 0 else 0
        d = _a.asx_raster_desc()
        d.rows, d.cols, d.edge_m = sc.rows, sc.cols, sc.l
        for s in range(4):
            d.bc[s] = int(sc.bc[s])
            d.free_begin[s], d.free_end[s] = (int(v) for v in sc.free_range[s])
        d.n_classes = nc
        d.max_samples = int(max_samples)
        d.cuda_stream = stream
        d.device = device
        d.precision = _a.ASX_FP64 if fp64 else _a.ASX_FP32_COMP
        self.desc = d
        self.handle = _a.asx_create_raster(d)
        self._keep = []
        self.set_params()
        shape = (sc.rows, sc.cols)
        theta = None if nc else _f32(sc.theta, shape)
        cls = np.ascontiguousarray(sc.cls.astype(np.uint8)) if nc else None
        _a.asx_set_fields(self.handle, _f64(sc.z, shape), theta, cls, _f32(sc.h0, shape),
                          _f32(sc.v1_0, shape), _f32(sc.v2_0, shape), _a.ASX_PTR_HOST)

    def set_params(self, cfl=None, dt_max=None, sample_dt=None):
        sc = self.sc
        p = _a.asx_params()
        p.g = sc.g
        p.cfl = sc.cfl if cfl is None else cfl
        p.dt_max = sc.dt_max if dt_max is None else dt_max
        p.viscosity = int(bool(getattr(sc, "viscosity", False)))
        p.tau = float(getattr(sc, "tau", 0.0))
        p.h_dry = float(getattr(sc, "h_dry", 0.0))
        for s in range(4):
            p.bc_q[s] = float(sc.bc_q[s])
            p.bc_h[s] = float(sc.bc_h[s])
            p.bc_u[s] = float(sc.bc_u[s])
        if self.desc.n_classes:
            ct = _f32(sc.class_theta, -1)
            cp = _f32(sc.class_alpha_p, -1)
            cs = _f32(sc.class_alpha_s, -1)
            self._keep += [ct, cp, cs]
            fp = C.POINTER(C.c_float)
            p.class_theta = ct.ctypes.data_as(fp)
            p.class_alpha_p = cp.ctypes.data_as(fp)
            p.class_alpha_s = cs.ctypes.data_as(fp)
        else:
            p.alpha_s = _uniform(sc.alpha_s, "alpha_s")
            p.alpha_p = _uniform(sc.alpha_p, "alpha_p")
        rt = np.ascontiguousarray(sc.rain_t, dtype=np.float64)
        rr = np.ascontiguousarray(sc.rain_r, dtype=np.float64)
        self._keep += [rt, rr]
        p.n_rain = int(rt.size)
        dp = C.POINTER(C.c_double)
        p.rain_t = rt.ctypes.data_as(dp)
        p.rain_r = rr.ctypes.data_as(dp)
        p.sample_dt = sc.sample_dt if sample_dt is None else sample_dt
        _a.asx_set_params(self.handle, p)

    # -- stepping
    def step(self, n=1):
        return _a.asx_step(self.handle, n)

    def run_until(self, t_end):
        return _a.asx_run_until(self.handle, t_end)

    # -- results
    def ledger(self):
        return _a.asx_mass_ledger(self.handle, 0)

    def clock(self):
        return _a.asx_get_clock(self.handle, 0)

    def fields(self):
        sh = (self.sc.rows, self.sc.cols)
        h, v1, v2 = (np.empty(sh, np.float32) for _ in range(3))
        _a.asx_get_fields(self.handle, 0, h, v1, v2, _a.ASX_PTR_HOST)
        return h, v1, v2

    def fields64(self):
        """Depth and velocity in float64 (the FP64 state, or the compensated float32 one)."""
        sh = (self.sc.rows, self.sc.cols)
        h, v1, v2 = (np.empty(sh, np.float64) for _ in range(3))
        _a.asx_get_fields64(self.handle, 0, h, v1, v2, _a.ASX_PTR_HOST)
        return h, v1, v2

    def state(self):
        sh = (self.sc.rows, self.sc.cols)
        mh, ml, v1, v2 = (np.empty(sh, np.float32) for _ in range(4))
        _a.asx_get_state(self.handle, mh, ml, v1, v2, _a.ASX_PTR_HOST)
        return mh, ml, v1, v2

    def mass64(self):
        mh, ml, v1, v2 = self.state()
        return mh.astype(np.float64) + ml.astype(np.float64), v1, v2

    def hydrograph(self, cap=1 << 20):
        return _a.asx_get_hydrograph(self.handle, 0, cap)[0]

    def close(self):
        if self.handle:
            _a.asx_destroy_raster(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
