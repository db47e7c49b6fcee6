"""Python access to the FP64 CPU oracle (``asx_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path (the CUDA
library and its binding) never imports this module.

The oracle is plain C compiled with gcc (strict IEEE double, no FMA contraction),
loaded through ctypes.  Arrays are numpy float64, row-major ``rows x cols``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SO_OMP = os.path.join(_BUILD, "liborc_omp.so")
_lock = threading.Lock()
_libs = {}

WALL, FREE = 0, 1
W, E, S, N = 0, 1, 2, 3
_CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def _compile(out, extra):
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *_CFLAGS, *extra, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborc.so`` (gcc, -O2, no FMA contraction)
    and its OpenMP build ``liborc_omp.so`` (the same source with -fopenmp: the cells of a
    step shared among threads, the same bits); returns the single-threaded library.

    ``ASX_ORACLE_SO`` names a prebuilt library to load instead (the mutation test uses it
    to run the pins against oracles with planted mistakes)."""
    if os.environ.get("ASX_ORACLE_SO"):
        return os.environ["ASX_ORACLE_SO"]
    os.makedirs(_BUILD, exist_ok=True)
    for out, extra in ((_SO, []), (_SO_OMP, ["-fopenmp"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
            _compile(out, extra)
    return _SO


def max_threads() -> int:
    """Cores this process may run on (the thread count the OpenMP build uses by default)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class _Problem(C.Structure):
    _fields_ = [("rows", C.c_int), ("cols", C.c_int), ("l", C.c_double), ("bc", C.c_int * 4),
                ("free_begin", C.c_int * 4), ("free_end", C.c_int * 4),
                ("g", C.c_double), ("cfl", C.c_double), ("dt_max", C.c_double),
                ("z", C.POINTER(C.c_double)), ("theta", C.POINTER(C.c_double)),
                ("alpha_s", C.POINTER(C.c_double)), ("alpha_p", C.POINTER(C.c_double)),
                ("n_rain", C.c_int), ("rain_t", C.POINTER(C.c_double)),
                ("rain_r", C.POINTER(C.c_double)), ("viscosity", C.c_int), ("tau", C.c_double),
                ("h_dry", C.c_double), ("bc_q", C.c_double * 4), ("bc_h", C.c_double * 4),
                ("bc_u", C.c_double * 4)]


class Ledger(C.Structure):
    _fields_ = [("rain_in", C.c_double), ("outflow", C.c_double), ("clamped", C.c_double),
                ("steps", C.c_longlong)]


def _load(threads: int = 1):
    """The oracle library: the single-threaded build for threads == 1, else the OpenMP
    build set to that many threads."""
    omp = threads > 1 and not os.environ.get("ASX_ORACLE_SO")
    with _lock:
        lib = _libs.get(omp)
        if lib is None:
            path = build()
            lib = C.CDLL(_SO_OMP if omp else path)
            dp = C.POINTER(C.c_double)
            P = C.POINTER(_Problem)
            lib.orc_step.argtypes = [P, dp, dp, dp, C.c_double, C.c_double, dp, dp, dp, C.POINTER(Ledger)]
            lib.orc_step.restype = C.c_int
            lib.orc_run.argtypes = [P, dp, dp, dp, dp, C.c_double, C.c_longlong, dp, C.c_longlong,
                                    C.c_double, dp, C.c_int, C.POINTER(C.c_int), C.POINTER(Ledger)]
            lib.orc_run.restype = C.c_longlong
            lib.orc_cfl_dt.argtypes = [P, dp, dp, dp]
            lib.orc_cfl_dt.restype = C.c_double
            lib.orc_cmax.argtypes = [P, dp, dp, dp]
            lib.orc_cmax.restype = C.c_double
            lib.orc_storage.argtypes = [P, dp]
            lib.orc_storage.restype = C.c_double
            lib.orc_rain_rate.argtypes = [P, C.c_double]
            lib.orc_rain_rate.restype = C.c_double
            lib.orc_friction.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, dp, dp]
            lib.orc_friction.restype = None
            lib.orc_sigma.argtypes = [C.c_double]
            lib.orc_sigma.restype = C.c_double
            lib.orc_phi.argtypes = [C.c_double]
            lib.orc_phi.restype = C.c_double
            lib.orc_neighbour.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.POINTER(C.c_int), C.POINTER(C.c_int)]
            lib.orc_neighbour.restype = C.c_int
            if hasattr(lib, "orc_threads"):
                lib.orc_threads.argtypes = [C.c_int]
                lib.orc_threads.restype = C.c_int
            _libs[omp] = lib
        if omp:
            lib.orc_threads(int(threads))
    return lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if a.size == 1 and n > 1:
        a = np.full(n, float(a[0]))
    assert a.size == n, (a.size, n)
    return a


class Problem:
    """Static data of one raster: geometry, boundary types, bed, porosity, coefficients, rain.
    ``threads`` > 1 runs steps on the OpenMP build of the oracle (bit-identical results)."""

    def __init__(self, rows, cols, l, z, theta, alpha_s, alpha_p, bc=(WALL, WALL, WALL, WALL),
                 g=9.81, cfl=0.5, dt_max=1.0, rain_t=(), rain_r=(), viscosity=False,
                 free_range=((0, 0), (0, 0), (0, 0), (0, 0)), tau=0.0, h_dry=0.0, bc_q=(0.0,) * 4,
                 bc_h=(0.0,) * 4, bc_u=(0.0,) * 4, threads=1):
        n = rows * cols
        self.threads = int(threads)
        self.rows, self.cols, self.l = int(rows), int(cols), float(l)
        self.z = _f64(z, n)
        self.theta = _f64(theta, n)
        self.alpha_s = _f64(alpha_s, n)
        self.alpha_p = _f64(alpha_p, n)
        self.rain_t = np.ascontiguousarray(np.asarray(rain_t, dtype=np.float64).reshape(-1))
        self.rain_r = np.ascontiguousarray(np.asarray(rain_r, dtype=np.float64).reshape(-1))
        assert self.rain_t.size == self.rain_r.size
        self.bc = tuple(int(b) for b in bc)
        self.free_range = tuple((int(a), int(b)) for a, b in free_range)
        self.g, self.cfl, self.dt_max = float(g), float(cfl), float(dt_max)
        self.viscosity = bool(viscosity)
        self.tau = float(tau)
        self.h_dry = float(h_dry)
        self.bc_q, self.bc_h, self.bc_u = (tuple(float(x) for x in v) for v in (bc_q, bc_h, bc_u))
        self._s = _Problem(self.rows, self.cols, self.l, (C.c_int * 4)(*self.bc),
                           (C.c_int * 4)(*[a for a, _ in self.free_range]),
                           (C.c_int * 4)(*[b for _, b in self.free_range]), self.g, self.cfl,
                           self.dt_max, _dp(self.z), _dp(self.theta), _dp(self.alpha_s),
                           _dp(self.alpha_p), int(self.rain_t.size), _dp(self.rain_t),
                           _dp(self.rain_r), int(self.viscosity), self.tau, self.h_dry,
                           (C.c_double * 4)(*self.bc_q), (C.c_double * 4)(*self.bc_h),
                           (C.c_double * 4)(*self.bc_u))

    @property
    def n(self):
        return self.rows * self.cols

    @property
    def sigma(self):
        return float(_load().orc_sigma(self.l))

    @property
    def phi(self):
        return float(_load().orc_phi(self.l))

    def mass(self, h):
        """theta*h from a depth field."""
        return _f64(h, self.n) * self.theta

    def depth(self, m):
        return _f64(m, self.n) / self.theta

    def rain_rate(self, t):
        return float(_load().orc_rain_rate(C.byref(self._s), float(t)))

    def cfl_dt(self, m, v1, v2):
        m, v1, v2 = (_f64(a, self.n) for a in (m, v1, v2))
        return float(_load(self.threads).orc_cfl_dt(C.byref(self._s), _dp(m), _dp(v1), _dp(v2)))

    def cmax(self, m, v1, v2):
        m, v1, v2 = (_f64(a, self.n) for a in (m, v1, v2))
        return float(_load(self.threads).orc_cmax(C.byref(self._s), _dp(m), _dp(v1), _dp(v2)))

    def storage(self, m):
        m = _f64(m, self.n)
        return float(_load().orc_storage(C.byref(self._s), _dp(m)))

    def neighbour(self, r, c, d):
        j, side = C.c_int(-1), C.c_int(-1)
        ok = _load().orc_neighbour(self.rows, self.cols, r, c, d, C.byref(j), C.byref(side))
        return (True, j.value) if ok else (False, side.value)

    def step(self, m, v1, v2, dt, t_next, ledger=None):
        """One step of Eq. fvm_2D_eq_frac.07; returns new (m, v1, v2)."""
        m, v1, v2 = (_f64(a, self.n) for a in (m, v1, v2))
        mo, ao, bo = np.empty(self.n), np.empty(self.n), np.empty(self.n)
        led = ledger if ledger is not None else Ledger()
        rc = _load(self.threads).orc_step(C.byref(self._s), _dp(m), _dp(v1), _dp(v2), float(dt), float(t_next),
                              _dp(mo), _dp(ao), _dp(bo), C.byref(led))
        if rc != 0:
            raise FloatingPointError("oracle step produced a non-finite value")
        return mo, ao, bo

    def run(self, m, v1, v2, t0, t_end, max_steps=1 << 62, t_replay=None, sample_dt=0.0,
            sample_cap=0, ledger=None):
        """Run to t_end.  Returns dict(m, v1, v2, t, steps, ledger, samples)."""
        m, v1, v2 = (_f64(a, self.n).copy() for a in (m, v1, v2))
        t = C.c_double(float(t0))
        led = ledger if ledger is not None else Ledger()
        samples = np.zeros(max(int(sample_cap), 1))
        ns = C.c_int(0)
        if t_replay is not None:
            rep = np.ascontiguousarray(np.asarray(t_replay, dtype=np.float64))
            rp, nr = _dp(rep), rep.size
        else:
            rp, nr = None, 0
        k = _load(self.threads).orc_run(C.byref(self._s), _dp(m), _dp(v1), _dp(v2), C.byref(t), float(t_end),
                            int(max_steps), rp, nr, float(sample_dt), _dp(samples), int(sample_cap),
                            C.byref(ns), C.byref(led))
        if k < 0:
            raise FloatingPointError("oracle run produced a non-finite value")
        return dict(m=m, v1=v1, v2=v2, t=t.value, steps=int(k), ledger=led,
                    samples=samples[:min(ns.value, int(sample_cap))].copy())


def from_scenario(sc, viscosity=None, threads=1):
    """Oracle problem for an ``inputs.Scenario`` (per-cell coefficient arrays); viscosity
    defaults to the scenario's setting."""
    if viscosity is None:
        viscosity = bool(getattr(sc, "viscosity", False))
    return Problem(sc.rows, sc.cols, sc.l, sc.z, sc.theta, sc.alpha_s, sc.alpha_p, bc=sc.bc,
                   g=sc.g, cfl=sc.cfl, dt_max=sc.dt_max, rain_t=sc.rain_t, rain_r=sc.rain_r,
                   viscosity=viscosity, free_range=sc.free_range, tau=getattr(sc, "tau", 0.0),
                   h_dry=getattr(sc, "h_dry", 0.0), bc_q=getattr(sc, "bc_q", (0.0,) * 4),
                   bc_h=getattr(sc, "bc_h", (0.0,) * 4), bc_u=getattr(sc, "bc_u", (0.0,) * 4),
                   threads=threads)


def friction(alpha, beta, g1, g2):
    """Closed-form implicit friction solve (Appendix A, Eq. miu-formula)."""
    a, b = C.c_double(), C.c_double()
    _load().orc_friction(float(alpha), float(beta), float(g1), float(g2), C.byref(a), C.byref(b))
    return a.value, b.value


def sigma(l):
    return float(_load().orc_sigma(float(l)))


def phi(l):
    return float(_load().orc_phi(float(l)))
