"""ctypes binding of the C ABI in ``include/asx.h`` (argument marshalling only).

Every function keeps its C name and raises ``AsxError`` on a non-zero status.  Device
buffers are passed as integer addresses (e.g. ``torch.Tensor.data_ptr()``), host buffers
as numpy arrays.  All computation happens in ``libasx.so``; if the library is missing
the import fails: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library this process loads: the in-tree build, or the file ASX_LIB names (e.g. the
# bounds-checked debug build, build.build_checked())
LIB_PATH = os.environ.get("ASX_LIB") or os.path.join(_HERE, "_build", "libasx.so")

ASX_OK, ASX_EINVAL, ASX_ENOMEM, ASX_ECUDA, ASX_ESTATE, ASX_ENUMERIC, ASX_ETIMEOUT, ASX_EBOUNDS = range(8)
STATUS_NAMES = {0: "ASX_OK", 1: "ASX_EINVAL", 2: "ASX_ENOMEM", 3: "ASX_ECUDA", 4: "ASX_ESTATE",
                5: "ASX_ENUMERIC", 6: "ASX_ETIMEOUT", 7: "ASX_EBOUNDS"}
ASX_BC_WALL, ASX_BC_FREE = 0, 1
ASX_SIDE_W, ASX_SIDE_E, ASX_SIDE_S, ASX_SIDE_N = 0, 1, 2, 3
ASX_PTR_HOST, ASX_PTR_DEVICE = 0, 1
ASX_FP32_COMP, ASX_FP64 = 0, 1
ASX_MAX_CLASSES = 16
ASX_MAX_RAIN = 64


class AsxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class asx_raster_desc(C.Structure):
    _fields_ = [("rows", C.c_int), ("cols", C.c_int), ("edge_m", C.c_double), ("bc", C.c_int * 4),
                ("free_begin", C.c_int * 4), ("free_end", C.c_int * 4), ("n_classes", C.c_int),
                ("max_samples", C.c_int), ("cuda_stream", C.c_void_p), ("device", C.c_int),
                ("precision", C.c_int)]


class asx_params(C.Structure):
    _fields_ = [("g", C.c_double), ("cfl", C.c_double), ("dt_max", C.c_double),
                ("alpha_s", C.c_double), ("alpha_p", C.c_double),
                ("class_theta", C.POINTER(C.c_float)), ("class_alpha_p", C.POINTER(C.c_float)),
                ("class_alpha_s", C.POINTER(C.c_float)), ("n_rain", C.c_int),
                ("rain_t", C.POINTER(C.c_double)), ("rain_r", C.POINTER(C.c_double)),
                ("sample_dt", C.c_double), ("viscosity", C.c_int), ("tau", C.c_double),
                ("h_dry", C.c_double), ("bc_q", C.c_double * 4), ("bc_h", C.c_double * 4),
                ("bc_u", C.c_double * 4)]


class asx_ledger(C.Structure):
    _fields_ = [("rain_in", C.c_double), ("outflow", C.c_double), ("storage", C.c_double),
                ("storage0", C.c_double), ("clamped", C.c_double), ("defect_rel", C.c_double),
                ("steps", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class asx_scenario_desc(C.Structure):
    _fields_ = [("rows", C.c_int), ("cols", C.c_int), ("edge_m", C.c_double), ("bc", C.c_int * 4),
                ("free_begin", C.c_int * 4), ("free_end", C.c_int * 4), ("g", C.c_double),
                ("cfl", C.c_double), ("dt_max", C.c_double), ("alpha_s", C.c_double),
                ("alpha_p", C.c_double), ("n_rain", C.c_int), ("rain_t", C.POINTER(C.c_double)),
                ("rain_r", C.POINTER(C.c_double)), ("t_end", C.c_double), ("sample_dt", C.c_double),
                ("max_samples", C.c_int), ("max_steps", C.c_longlong), ("bc_q", C.c_double * 4),
                ("bc_h", C.c_double * 4), ("bc_u", C.c_double * 4), ("viscosity", C.c_int),
                ("tau", C.c_double), ("h_dry", C.c_double)]


class asx_ensemble_tuning(C.Structure):
    _fields_ = [("cluster", C.c_int), ("threads", C.c_int), ("cells_per_thread", C.c_int), ("tile_rows", C.c_int),
                ("split", C.c_int)]

    def as_tuple(self):
        return (self.cluster, self.threads, self.cells_per_thread, self.tile_rows, self.split)


_vp = C.c_void_p
_RASTER = C.c_void_p
_ENS = C.c_void_p

# name: (restype, argtypes)
_PROTOS = {
    "asx_create_raster": (C.c_int, [C.POINTER(asx_raster_desc), C.POINTER(_RASTER)]),
    "asx_destroy_raster": (C.c_int, [_RASTER]),
    "asx_set_params": (C.c_int, [_RASTER, C.POINTER(asx_params)]),
    "asx_set_fields": (C.c_int, [_RASTER, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int]),
    "asx_step": (C.c_int, [_RASTER, C.c_int, C.POINTER(C.c_double)]),
    "asx_run_until": (C.c_int, [_RASTER, C.c_double, C.POINTER(C.c_double)]),
    "asx_mass_ledger": (C.c_int, [_RASTER, C.c_int, C.POINTER(asx_ledger)]),
    "asx_get_fields": (C.c_int, [_RASTER, C.c_int, _vp, _vp, _vp, C.c_int]),
    "asx_get_fields64": (C.c_int, [_RASTER, C.c_int, _vp, _vp, _vp, C.c_int]),
    "asx_get_state": (C.c_int, [_RASTER, _vp, _vp, _vp, _vp, C.c_int]),
    "asx_set_state": (C.c_int, [_RASTER, _vp, _vp, _vp, _vp, C.c_int, C.c_double, C.c_longlong,
                                C.POINTER(asx_ledger), C.c_int, _vp]),
    "asx_get_hydrograph": (C.c_int, [_RASTER, C.c_int, _vp, C.c_int, C.POINTER(C.c_int)]),
    "asx_get_clock": (C.c_int, [_RASTER, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                C.POINTER(C.c_longlong)]),
    "asx_last_error": (C.c_char_p, [_RASTER]),
    "asx_selftest_wait": (C.c_int, [C.c_int]),
    "asx_state_scan_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _vp, _vp,
                                         _vp, _vp, _vp, _vp, _vp, _vp]),
    "asx_create_ensemble": (C.c_int, [C.c_int, C.POINTER(asx_scenario_desc), _vp, C.c_int, C.POINTER(_ENS)]),
    "asx_destroy_ensemble": (C.c_int, [_ENS]),
    "asx_ensemble_set_fields": (C.c_int, [_ENS, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_int]),
    "asx_ensemble_autotune": (C.c_int, [_ENS, C.c_int, C.POINTER(asx_ensemble_tuning)]),
    "asx_ensemble_run": (C.c_int, [_ENS, C.POINTER(asx_ensemble_tuning)]),
    "asx_ensemble_ledger": (C.c_int, [_ENS, C.c_int, C.POINTER(asx_ledger)]),
    "asx_ensemble_get_fields": (C.c_int, [_ENS, C.c_int, _vp, _vp, _vp, C.c_int]),
    "asx_ensemble_get_state": (C.c_int, [_ENS, C.c_int, _vp, _vp, _vp, _vp, C.c_int]),
    "asx_ensemble_get_hydrograph": (C.c_int, [_ENS, C.c_int, _vp, C.c_int, C.POINTER(C.c_int)]),
    "asx_ensemble_get_clock": (C.c_int, [_ENS, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "asx_ensemble_last_error": (C.c_char_p, [_ENS]),
    "asx_gemm_bf16": (C.c_int, [C.c_int, C.c_int, C.c_int, _vp, C.c_longlong, C.c_longlong, _vp, C.c_longlong,
                                C.c_longlong, _vp, C.c_longlong, _vp]),
    "asx_mlp_create": (C.c_int, [C.c_int, _vp, C.c_int, C.POINTER(_vp)]),
    "asx_mlp_destroy": (C.c_int, [_vp]),
    "asx_mlp_set_params": (C.c_int, [_vp, _vp, C.c_int]),
    "asx_mlp_get_params": (C.c_int, [_vp, _vp, C.c_int]),
    "asx_mlp_forward": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int]),
    "asx_mlp_gradients": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.POINTER(C.c_float), C.c_int]),
    "asx_mlp_train_step": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_float, C.c_float, C.POINTER(C.c_float),
                                     C.c_int]),
    "asx_mlp_last_error": (C.c_char_p, [_vp]),
    "asx_surrogate_check": (C.c_int, [C.c_int, C.c_int, _vp, _vp, _vp, C.c_float, _vp, _vp, _vp]),
}

ASX_MLP_IN, ASX_MLP_HIDDEN, ASX_MLP_OUT, ASX_MLP_PARAMS = 36, 256, 128, 173952

_lib = None


def load(path: str = LIB_PATH):
    """Load libasx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2406_14933_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_names():
    return list(_PROTOS)


def _check(st, r=None):
    if st != ASX_OK:
        msg = load().asx_last_error(r).decode() if r else ""
        raise AsxError(st, msg)


def _ptr(x):
    """Address of a numpy array, an integer device address, a torch tensor, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(type(x))


# ----------------------------------------------------------------- C-named wrappers

def asx_create_raster(desc: asx_raster_desc):
    r = _RASTER()
    _check(load().asx_create_raster(C.byref(desc), C.byref(r)))
    return r


def asx_destroy_raster(r):
    _check(load().asx_destroy_raster(r))


def asx_set_params(r, p: asx_params):
    _check(load().asx_set_params(r, C.byref(p)), r)


def _dtype_is(x, name, want):
    """Refuses a host or torch array whose element type differs from the C signature's
    (the library would read its bytes as the other type)."""
    if x is None or isinstance(x, int):
        return
    dt = getattr(x, "dtype", None)
    got = str(dt).replace("torch.", "") if dt is not None else None
    if got is not None and got != want:
        raise TypeError(f"{name} must be {want}, got {got}")


def asx_set_fields(r, z, theta, cls, h0, v1, v2, ptr_kind):
    _dtype_is(z, "z", "float64")
    for nm, x in (("theta", theta), ("h0", h0), ("v1", v1), ("v2", v2)):
        _dtype_is(x, nm, "float32")
    _dtype_is(cls, "cls", "uint8")
    _check(load().asx_set_fields(r, _ptr(z), _ptr(theta), _ptr(cls), _ptr(h0), _ptr(v1), _ptr(v2),
                                 ptr_kind), r)


def asx_step(r, n_steps):
    t = C.c_double()
    _check(load().asx_step(r, int(n_steps), C.byref(t)), r)
    return t.value


def asx_run_until(r, t_end):
    t = C.c_double()
    _check(load().asx_run_until(r, float(t_end), C.byref(t)), r)
    return t.value


def asx_mass_ledger(r, scenario=0):
    led = asx_ledger()
    _check(load().asx_mass_ledger(r, int(scenario), C.byref(led)), r)
    return led


def asx_get_fields(r, scenario, h, v1, v2, ptr_kind):
    _check(load().asx_get_fields(r, int(scenario), _ptr(h), _ptr(v1), _ptr(v2), ptr_kind), r)


def asx_get_fields64(r, scenario, h, v1, v2, ptr_kind):
    _check(load().asx_get_fields64(r, int(scenario), _ptr(h), _ptr(v1), _ptr(v2), ptr_kind), r)


def asx_get_state(r, m_hi, m_lo, v1, v2, ptr_kind):
    _check(load().asx_get_state(r, _ptr(m_hi), _ptr(m_lo), _ptr(v1), _ptr(v2), ptr_kind), r)


def asx_set_state(r, m_hi, m_lo, v1, v2, ptr_kind, t, step, ledger, samples=None):
    ns = 0 if samples is None else int(len(samples))
    sp = None if samples is None else _ptr(np.ascontiguousarray(samples, dtype=np.float64))
    keep = samples
    _check(load().asx_set_state(r, _ptr(m_hi), _ptr(m_lo), _ptr(v1), _ptr(v2), ptr_kind, float(t),
                                int(step), C.byref(ledger), ns, sp), r)
    del keep


def asx_get_hydrograph(r, scenario, cap):
    q = np.zeros(max(int(cap), 1))
    n = C.c_int()
    _check(load().asx_get_hydrograph(r, int(scenario), q.ctypes.data, int(cap), C.byref(n)), r)
    return q[:min(n.value, int(cap))].copy(), n.value


def asx_get_clock(r, scenario=0):
    t, dt, s = C.c_double(), C.c_double(), C.c_longlong()
    _check(load().asx_get_clock(r, int(scenario), C.byref(t), C.byref(dt), C.byref(s)), r)
    return t.value, dt.value, s.value


def asx_last_error(r):
    return load().asx_last_error(r).decode()


def asx_state_scan_noalloc(rows, cols, pitch, edge_m, g, m_hi, m_lo, v1, v2, theta, storage_out,
                           cmax_out, cuda_stream=None):
    """Allocation-free storage / wave-speed scan of a caller-held device state (see asx.h);
    every pointer is a device address, the outputs are written asynchronously."""
    _check(load().asx_state_scan_noalloc(int(rows), int(cols), int(pitch), float(edge_m), float(g),
                                         _ptr(m_hi), _ptr(m_lo), _ptr(v1), _ptr(v2), _ptr(theta),
                                         _ptr(storage_out), _ptr(cmax_out), cuda_stream))


def asx_selftest_wait(device=0):
    """Runs the bounded-wait self-test (see asx.h) and returns its status code: ASX_ETIMEOUT
    when the timeout was detected and reported."""
    return load().asx_selftest_wait(int(device))


# ----------------------------------------------------------------- ensembles

def _echeck(st, e=None):
    if st != ASX_OK:
        msg = load().asx_ensemble_last_error(e).decode() if e else ""
        raise AsxError(st, msg)


def asx_create_ensemble(descs, cuda_stream=None, device=0):
    arr = (asx_scenario_desc * len(descs))(*descs)
    e = _ENS()
    _echeck(load().asx_create_ensemble(len(descs), arr, cuda_stream, int(device), C.byref(e)))
    return e


def asx_destroy_ensemble(e):
    _echeck(load().asx_destroy_ensemble(e))


def asx_ensemble_set_fields(e, s, z, theta, h0, v1, v2, ptr_kind):
    _dtype_is(z, "z", "float64")
    for nm, x in (("theta", theta), ("h0", h0), ("v1", v1), ("v2", v2)):
        _dtype_is(x, nm, "float32")
    _echeck(load().asx_ensemble_set_fields(e, int(s), _ptr(z), _ptr(theta), _ptr(h0), _ptr(v1), _ptr(v2),
                                           ptr_kind), e)


def asx_ensemble_autotune(e, max_steps):
    t = asx_ensemble_tuning()
    _echeck(load().asx_ensemble_autotune(e, int(max_steps), C.byref(t)), e)
    return t


def asx_ensemble_run(e, tuning=None):
    _echeck(load().asx_ensemble_run(e, C.byref(tuning) if tuning is not None else None), e)


def asx_ensemble_ledger(e, s):
    led = asx_ledger()
    _echeck(load().asx_ensemble_ledger(e, int(s), C.byref(led)), e)
    return led


def asx_ensemble_get_fields(e, s, h, v1, v2, ptr_kind):
    _echeck(load().asx_ensemble_get_fields(e, int(s), _ptr(h), _ptr(v1), _ptr(v2), ptr_kind), e)


def asx_ensemble_get_state(e, s, m_hi, m_lo, v1, v2, ptr_kind):
    _echeck(load().asx_ensemble_get_state(e, int(s), _ptr(m_hi), _ptr(m_lo), _ptr(v1), _ptr(v2), ptr_kind), e)


def asx_ensemble_get_hydrograph(e, s, cap):
    q = np.zeros(max(int(cap), 1))
    n = C.c_int()
    _echeck(load().asx_ensemble_get_hydrograph(e, int(s), q.ctypes.data, int(cap), C.byref(n)), e)
    return q[:min(n.value, int(cap))].copy(), n.value


def asx_ensemble_get_clock(e, s):
    t, k = C.c_double(), C.c_longlong()
    _echeck(load().asx_ensemble_get_clock(e, int(s), C.byref(t), C.byref(k)), e)
    return t.value, k.value


def asx_ensemble_last_error(e):
    return load().asx_ensemble_last_error(e).decode()


def asx_gemm_bf16(M, N, K, A, sam, sak, B, sbn, sbk, D, ldd, cuda_stream=None):
    """Tensor-core GEMM D = A . B^T (BF16 in, FP32 out), device pointers (see asx.h)."""
    _check(load().asx_gemm_bf16(int(M), int(N), int(K), _ptr(A), int(sam), int(sak), _ptr(B), int(sbn),
                                int(sbk), _ptr(D), int(ldd), cuda_stream))


# ----------------------------------------------------------------- the surrogate MLP

def _mcheck(st, p=None):
    if st != ASX_OK:
        msg = load().asx_mlp_last_error(p).decode() if p else ""
        raise AsxError(st, msg)


def asx_mlp_create(device=0, cuda_stream=None, max_batch=65536):
    p = _vp()
    _mcheck(load().asx_mlp_create(int(device), cuda_stream, int(max_batch), C.byref(p)))
    return p


def asx_mlp_destroy(p):
    _mcheck(load().asx_mlp_destroy(p))


def asx_mlp_set_params(p, params, ptr_kind=ASX_PTR_HOST):
    _mcheck(load().asx_mlp_set_params(p, _ptr(params), ptr_kind), p)


def asx_mlp_get_params(p, params, ptr_kind=ASX_PTR_HOST):
    _mcheck(load().asx_mlp_get_params(p, _ptr(params), ptr_kind), p)


def asx_mlp_forward(p, batch, x, y, ptr_kind=ASX_PTR_HOST):
    _mcheck(load().asx_mlp_forward(p, int(batch), _ptr(x), _ptr(y), ptr_kind), p)


def asx_mlp_gradients(p, batch, x, t, grad, ptr_kind=ASX_PTR_HOST):
    loss = C.c_float()
    _mcheck(load().asx_mlp_gradients(p, int(batch), _ptr(x), _ptr(t), _ptr(grad), C.byref(loss), ptr_kind), p)
    return loss.value


def asx_mlp_train_step(p, batch, x, t, lr, weight_decay=0.0, ptr_kind=ASX_PTR_HOST, want_loss=True):
    loss = C.c_float()
    _mcheck(load().asx_mlp_train_step(p, int(batch), _ptr(x), _ptr(t), float(lr), float(weight_decay),
                                      C.byref(loss) if want_loss else None, ptr_kind), p)
    return loss.value if want_loss else None


def asx_mlp_last_error(p):
    return load().asx_mlp_last_error(p).decode()


def asx_surrogate_check(batch, n_check, idx, y, ref, tol, rel_err, n_replaced, cuda_stream=None):
    """All array arguments are device pointers (ints) or CUDA tensors."""
    _check(load().asx_surrogate_check(int(batch), int(n_check), _ptr(idx), _ptr(y), _ptr(ref), float(tol),
                                      _ptr(rel_err), _ptr(n_replaced), cuda_stream))
