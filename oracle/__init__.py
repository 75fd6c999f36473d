"""FP64 CPU oracle for the CETRA transit search (Smith et al. 2025, Sec. 2).

TEST INFRASTRUCTURE ONLY. This package is imported by the test suite, by the
smoke check of the build entry point and by the benchmark's CPU-baseline leg,
and by nothing else. The product (the CUDA library and its Python binding)
never imports, links or calls it, and the two share no code.

The arithmetic lives in ``cetra_oracle.c`` (plain C, FP64, OpenMP over
independent windows / periods); this module only builds it and marshals numpy
arrays through ctypes. Each C function cites the passage of the paper it
follows and lists the readings taken where the paper is silent.

Parity status: every step is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (closed forms, noiseless injections, brute-force
likelihood maximisation, invariants, the paper's toy example); the only
conventions that no external fact fixes are the readings R1, R3, R5, R6 and R7
listed in the C file, which are choices rather than results (parity unpinned for
those conventions only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cetra_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc, FP64, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", _LIB + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Geom(ctypes.Structure):
    _fields_ = [
        ("t_ref", ctypes.c_double),
        ("cadence", ctypes.c_double),
        ("t0_step", ctypes.c_double),
        ("p", ctypes.c_int64),
        ("q", ctypes.c_int64),
        ("n_pad", ctypes.c_int64),
        ("n_grid", ctypes.c_int64),
        ("n_t0", ctypes.c_int64),
        ("n_kept", ctypes.c_int64),
        ("tau_max", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    lib.oracle_geometry.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    P, ctypes.c_int, ctypes.POINTER(_Geom)]
    lib.oracle_resample.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int,
                                    ctypes.POINTER(_Geom), P, P]
    lib.oracle_template.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
    lib.oracle_linear.argtypes = [ctypes.POINTER(_Geom), P, P, P, ctypes.c_int, P, ctypes.c_int,
                                  P, P, P, P]
    lib.oracle_periodic.argtypes = [ctypes.POINTER(_Geom), P, ctypes.c_int, P, P, P, P,
                                    ctypes.c_int, P, P, P, P, P, P, P, P]
    lib.oracle_linear_cells.argtypes = [ctypes.POINTER(_Geom), P, P, P, ctypes.c_int, P,
                                        ctypes.c_int, ctypes.c_int64, P, P, P, P, P, P]
    lib.oracle_periodic_at.argtypes = [ctypes.POINTER(_Geom), ctypes.c_int, P, P, P, P,
                                       ctypes.c_int, P, P, P, P, P]
    lib.oracle_logl0.argtypes = [ctypes.POINTER(_Geom), P, P]
    lib.oracle_period_grid.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int64, P]
    lib.oracle_period_grid.restype = ctypes.c_int64
    lib.oracle_logl0.restype = ctypes.c_double
    lib.oracle_mask_transits.argtypes = [ctypes.POINTER(_Geom), P, P, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double]
    lib.oracle_mask_transits.restype = ctypes.c_int64
    lib.oracle_monotransits.argtypes = [ctypes.POINTER(_Geom), P, ctypes.c_int, P, P,
                                        ctypes.c_int, P, P]
    lib.oracle_monotransits.restype = ctypes.c_int
    lib.oracle_num_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


@dataclass
class Geometry:
    t_ref: float
    cadence: float
    t0_step: float
    p: int
    q: int
    n_pad: int
    n_grid: int
    n_t0: int
    n_kept: int
    tau_max: float
    _raw: _Geom = None


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def geometry(time, flux, flux_err, durations, cadence=0.0, t0_step=0.0) -> Geometry:
    lib = _load()
    t = np.ascontiguousarray(time, np.float64)
    f = np.ascontiguousarray(flux, np.float32)
    e = np.ascontiguousarray(flux_err, np.float32)
    d = np.ascontiguousarray(durations, np.float64)
    g = _Geom()
    _check(lib.oracle_geometry(_ptr(t), _ptr(f), _ptr(e), t.size, float(cadence), float(t0_step),
                               _ptr(d), d.size, ctypes.byref(g)), "geometry")
    return Geometry(g.t_ref, g.cadence, g.t0_step, g.p, g.q, g.n_pad, g.n_grid, g.n_t0,
                    g.n_kept, g.tau_max, g)


def resample(time, flux, flux_err, geom: Geometry, flux_is_offset=False):
    lib = _load()
    t = np.ascontiguousarray(time, np.float64)
    f = np.ascontiguousarray(flux, np.float32)
    e = np.ascontiguousarray(flux_err, np.float32)
    y = np.empty(geom.n_grid, np.float64)
    w = np.empty(geom.n_grid, np.float64)
    _check(lib.oracle_resample(_ptr(t), _ptr(f), _ptr(e), t.size, int(bool(flux_is_offset)),
                               ctypes.byref(geom._raw), _ptr(y), _ptr(w)), "resample")
    return y, w


def template(tmpl, L=1024):
    lib = _load()
    tm = np.ascontiguousarray(tmpl, np.float32)
    out = np.empty(int(L), np.float64)
    _check(lib.oracle_template(_ptr(tm), tm.size, int(L), _ptr(out)), "template")
    return out


def linear(geom: Geometry, y_grid, w_grid, durations, T, with_kappa=False):
    """Linear search (Sec. 2.2). Returns depth, depth_var, LR (and kappa), each [J][I]."""
    lib = _load()
    y = np.ascontiguousarray(y_grid, np.float64)
    w = np.ascontiguousarray(w_grid, np.float64)
    d = np.ascontiguousarray(durations, np.float64)
    Tm = np.ascontiguousarray(T, np.float64)
    J, I = d.size, geom.n_t0
    dep = np.empty((J, I), np.float64)
    var = np.empty((J, I), np.float64)
    lr = np.empty((J, I), np.float64)
    kap = np.empty((J, I), np.float64) if with_kappa else None
    _check(lib.oracle_linear(ctypes.byref(geom._raw), _ptr(y), _ptr(w), _ptr(d), J, _ptr(Tm),
                             Tm.size, _ptr(dep), _ptr(var), _ptr(lr), _ptr(kap)), "linear")
    if with_kappa:
        return dep, var, lr, kap
    return dep, var, lr


def linear_cells(geom: Geometry, y_grid, w_grid, durations, T, j, i):
    """Linear search at the cells (j[c], i[c]) only. Returns depth, depth_var, LR, kappa."""
    lib = _load()
    y = np.ascontiguousarray(y_grid, np.float64)
    w = np.ascontiguousarray(w_grid, np.float64)
    d = np.ascontiguousarray(durations, np.float64)
    Tm = np.ascontiguousarray(T, np.float64)
    jj = np.ascontiguousarray(j, np.int32)
    ii = np.ascontiguousarray(i, np.int64)
    n = jj.size
    out = [np.empty(n, np.float64) for _ in range(4)]
    _check(lib.oracle_linear_cells(ctypes.byref(geom._raw), _ptr(y), _ptr(w), _ptr(d), d.size,
                                   _ptr(Tm), Tm.size, n, _ptr(jj), _ptr(ii), *[_ptr(o) for o in out]),
           "linear_cells")
    return tuple(out)


def periodic_at(geom: Geometry, depth, depth_var, lr, periods, i_at, j_at):
    """Eq. 4 at (i_at[k], j_at[k]) for each period k. Returns LR, Z, var_Z."""
    lib = _load()
    dep = np.ascontiguousarray(depth, np.float64)
    var = np.ascontiguousarray(depth_var, np.float64)
    l = np.ascontiguousarray(lr, np.float64)
    P = np.ascontiguousarray(periods, np.float64)
    ii = np.ascontiguousarray(i_at, np.int64)
    jj = np.ascontiguousarray(j_at, np.int32)
    out = [np.empty(P.size, np.float64) for _ in range(3)]
    _check(lib.oracle_periodic_at(ctypes.byref(geom._raw), dep.shape[0], _ptr(dep), _ptr(var),
                                  _ptr(l), _ptr(P), P.size, _ptr(ii), _ptr(jj),
                                  *[_ptr(o) for o in out]), "periodic_at")
    return tuple(out)


def periodic(geom: Geometry, durations, depth, depth_var, lr, periods, mask=None):
    """Periodic search (Sec. 2.3). Returns a dict of per-period arrays."""
    lib = _load()
    d = np.ascontiguousarray(durations, np.float64)
    P = np.ascontiguousarray(periods, np.float64)
    dep = np.ascontiguousarray(depth, np.float64)
    var = np.ascontiguousarray(depth_var, np.float64)
    l = np.ascontiguousarray(lr, np.float64)
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    K = P.size
    out = {k: np.empty(K, np.float64) for k in ("dlogl", "t0", "duration", "depth", "depth_var")}
    out["i"] = np.empty(K, np.int64)
    out["j"] = np.empty(K, np.int32)
    _check(lib.oracle_periodic(ctypes.byref(geom._raw), _ptr(d), d.size, _ptr(dep), _ptr(var),
                               _ptr(l), _ptr(P), K, _ptr(m), _ptr(out["dlogl"]), _ptr(out["t0"]),
                               _ptr(out["duration"]), _ptr(out["depth"]),
                               _ptr(out["depth_var"]), _ptr(out["i"]), _ptr(out["j"])),
           "periodic")
    return out


def period_grid(pmin, ratio, pmax):
    """The batched search's period grid: pmin * ratio^k (square-and-multiply) up to pmax."""
    lib = _load()
    n = lib.oracle_period_grid(float(pmin), float(ratio), float(pmax), 0, None)
    if n < 0:
        raise ValueError("bad period grid")
    out = np.empty(n, np.float64)
    lib.oracle_period_grid(float(pmin), float(ratio), float(pmax), n, _ptr(out))
    return out


def logl0(geom: Geometry, y_grid, w_grid) -> float:
    lib = _load()
    y = np.ascontiguousarray(y_grid, np.float64)
    w = np.ascontiguousarray(w_grid, np.float64)
    return float(lib.oracle_logl0(ctypes.byref(geom._raw), _ptr(y), _ptr(w)))


def search(time, flux, flux_err, durations, tmpl, periods=None, *, cadence=0.0, t0_step=0.0,
           L=1024, flux_is_offset=False, mask=None, with_kappa=False):
    """Whole pipeline: geometry, resample, template, linear search and (optionally) periodic."""
    g = geometry(time, flux, flux_err, durations, cadence, t0_step)
    y, w = resample(time, flux, flux_err, g, flux_is_offset)
    T = template(tmpl, L)
    lin = linear(g, y, w, durations, T, with_kappa=with_kappa)
    res = {"geom": g, "y_grid": y, "w_grid": w, "T": T, "depth": lin[0], "depth_var": lin[1],
           "dlogl": lin[2]}
    if with_kappa:
        res["kappa"] = lin[3]
    res["logl0"] = logl0(g, y, w)
    if periods is not None:
        res["periodic"] = periodic(g, durations, lin[0], lin[1], lin[2], periods, mask)
    return res


def mask_transits(geom: Geometry, y_grid, w_grid, period, t0, half_width):
    """R17: copies of (y, w) with the cells within half_width days of any mid-time
    t0 + n period nulled, and the number of non-null cells that were nulled."""
    lib = _load()
    y = np.array(y_grid, np.float64, copy=True)
    w = np.array(w_grid, np.float64, copy=True)
    n = lib.oracle_mask_transits(ctypes.byref(geom._raw), _ptr(y), _ptr(w), float(period),
                                 float(t0), float(half_width))
    return y, w, int(n)


def monotransits(geom: Geometry, durations, depth, lr, max_events):
    """R18: (i, j) of up to max_events single-transit events, strongest first."""
    lib = _load()
    d = np.ascontiguousarray(durations, np.float64)
    dep = np.ascontiguousarray(depth, np.float64)
    l = np.ascontiguousarray(lr, np.float64)
    ii = np.empty(max(1, max_events), np.int64)
    jj = np.empty(max(1, max_events), np.int32)
    n = lib.oracle_monotransits(ctypes.byref(geom._raw), _ptr(d), d.size, _ptr(dep), _ptr(l),
                                int(max_events), _ptr(ii), _ptr(jj))
    if n < 0:
        raise MemoryError("oracle monotransits")
    return ii[:n].copy(), jj[:n].copy()


def t0_of(geom: Geometry, i):
    """Mid-time of t0 index i: t_ref + (i p - n_pad q) c / q."""
    return geom.t_ref + ((float(i * geom.p - geom.n_pad * geom.q)) * geom.cadence) / float(geom.q)


def search_iterative(time, flux, flux_err, durations, tmpl, periods, n_iter, width=2.0, *,
                     cadence=0.0, t0_step=0.0, L=1024, mask=None):
    """Sec. 4.2 with R17: search, null the cells within width/2 durations of the best
    signal's mid-times, search again; n_iter detections (fewer if a search finds nothing).
    Each detection: dict(k, period, t0, duration, depth, depth_var, dlogl, i, j)."""
    g = geometry(time, flux, flux_err, durations, cadence, t0_step)
    y, w = resample(time, flux, flux_err, g)
    T = template(tmpl, L)
    P = np.ascontiguousarray(periods, np.float64)
    out = []
    for r in range(n_iter):
        dep, var, lr = linear(g, y, w, durations, T)
        per = periodic(g, durations, dep, var, lr, P, mask)
        if np.all(np.isnan(per["dlogl"])):
            break
        k = int(np.nanargmax(per["dlogl"]))
        det = dict(k=k, period=float(P[k]), t0=float(per["t0"][k]),
                   duration=float(per["duration"][k]), depth=float(per["depth"][k]),
                   depth_var=float(per["depth_var"][k]), dlogl=float(per["dlogl"][k]),
                   i=int(per["i"][k]), j=int(per["j"][k]), lr=per["dlogl"], linear=(dep, var, lr))
        out.append(det)
        if r + 1 < n_iter:
            y, w, _ = mask_transits(g, y, w, det["period"], det["t0"], 0.5 * width * det["duration"])
    return out, g
