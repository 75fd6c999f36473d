"""ctypes binding of libcetra.so: the C ABI of include/cetra.h under the same names.

Argument marshalling only. The library is built in-tree (``build.py``); if it
is missing this module raises at import time rather than falling back to any
other implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcetra.so")

CETRA_OK = 0
CETRA_EINVAL = 1
CETRA_ENOMEM = 2
CETRA_ECUDA = 3
CETRA_ETIMEOUT = 4
CETRA_ECAPACITY = 5
CETRA_FP32 = 0
CETRA_FP32_KAHAN = 1
CETRA_STATIC_MAX_PERIODS = 262144  # periods the allocation-free entry point accepts

STATUS_NAMES = {0: "CETRA_OK", 1: "CETRA_EINVAL", 2: "CETRA_ENOMEM", 3: "CETRA_ECUDA",
                4: "CETRA_ETIMEOUT", 5: "CETRA_ECAPACITY"}


class cetra_params(ctypes.Structure):
    _fields_ = [("cadence", ctypes.c_double), ("t0_step", ctypes.c_double),
                ("template_samples", ctypes.c_int), ("flux_is_offset", ctypes.c_int),
                ("precision", ctypes.c_int)]


class cetra_plan_info(ctypes.Structure):
    _fields_ = [("t_ref", ctypes.c_double), ("cadence", ctypes.c_double),
                ("t0_step", ctypes.c_double), ("p", ctypes.c_int64), ("q", ctypes.c_int64),
                ("n_pad", ctypes.c_int64), ("n_grid", ctypes.c_int64), ("n_t0", ctypes.c_int64),
                ("n_kept", ctypes.c_int64), ("n_dur", ctypes.c_int32),
                ("template_samples", ctypes.c_int32), ("table_entries", ctypes.c_int64),
                ("grid_bytes", ctypes.c_size_t)]


class cetra_best(ctypes.Structure):
    _fields_ = [("dlogl", ctypes.c_double), ("period", ctypes.c_double), ("t0", ctypes.c_double),
                ("duration", ctypes.c_double), ("depth", ctypes.c_double),
                ("depth_var", ctypes.c_double), ("k", ctypes.c_int64), ("i", ctypes.c_int64),
                ("j", ctypes.c_int32), ("n_periods", ctypes.c_int32)]


class cetra_event(ctypes.Structure):
    _fields_ = [("dlogl", ctypes.c_double), ("t0", ctypes.c_double),
                ("duration", ctypes.c_double), ("depth", ctypes.c_double),
                ("depth_var", ctypes.c_double), ("i", ctypes.c_int64), ("j", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class cetra_batch_info(ctypes.Structure):
    _fields_ = [("n_curves", ctypes.c_int32), ("n_dur", ctypes.c_int32),
                ("n_points", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("n_t0", ctypes.c_int64), ("n_periods", ctypes.c_int64),
                ("n_fold_items", ctypes.c_int64), ("fold_cell_reads", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("linear_threads", ctypes.c_int32),
                ("fold_variant", ctypes.c_int32), ("fold_blocks", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("cadence", ctypes.c_double),
                ("t0_step", ctypes.c_double), ("p", ctypes.c_int64), ("q", ctypes.c_int64),
                ("n_pad", ctypes.c_int64)]


class CetraError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int
_SZ = ctypes.c_size_t

# name -> (restype, argtypes)
SIGNATURES = {
    "cetra_params_default": (None, [ctypes.POINTER(cetra_params)]),
    "cetra_create": (_INT, [ctypes.POINTER(_P), _INT, _P]),
    "cetra_destroy": (None, [_P]),
    "cetra_set_stream": (_INT, [_P, _P]),
    "cetra_last_error": (ctypes.c_char_p, [_P]),
    "cetra_kernel_launches": (_I64, [_P]),
    "cetra_profile_enable": (_INT, [_P, _INT]),
    "cetra_profile_read": (_INT, [_P, ctypes.c_char_p, ctypes.POINTER(_I64),
                                  ctypes.POINTER(ctypes.c_double)]),
    "cetra_plan_create": (_INT, [_P, ctypes.POINTER(cetra_params), _P, _P, _P, _I64, _P, _INT,
                                 _P, _INT, ctypes.POINTER(_P)]),
    "cetra_plan_get_info": (_INT, [_P, ctypes.POINTER(cetra_plan_info)]),
    "cetra_plan_geometry": (_INT, [_P, ctypes.POINTER(cetra_params), _P, _P, _P, _I64, _P, _INT,
                                   ctypes.POINTER(cetra_plan_info)]),
    "cetra_plan_destroy": (None, [_P]),
    "cetra_workspace_bytes": (_SZ, [_P, _INT]),
    "cetra_resample_device": (_INT, [_P, _P, _P, _P, _P, _I64, _P, _SZ]),
    "cetra_linear_device": (_INT, [_P, _P, _P, _SZ, _P, _P, _P]),
    "cetra_periodic_device": (_INT, [_P, _P, _P, _SZ, _P, _INT, _P, _P, _P, _P, _P, _P, _P,
                                     _P]),
    "cetra_logl0_device": (_INT, [_P, _P, _P, _SZ, _P]),
    "cetra_workspace_status": (_INT, [_P, _P, _P, _SZ, ctypes.POINTER(_INT)]),
    "cetra_periodic_device_static": (_INT, [_P, _P, _P, _SZ, _P, _INT, _P, _P, _P, _P, _P, _P,
                                            _P, _P]),
    "cetra_static_status": (_INT, [_P, ctypes.POINTER(_INT)]),
    "cetra_selftest_static_timeout": (_INT, [_P]),
    "cetra_linear_search": (_INT, [_P, ctypes.POINTER(cetra_params), _P, _P, _P, _I64, _P, _INT,
                                   _P, _INT, ctypes.POINTER(_P), _P, _P, _P,
                                   ctypes.POINTER(_I64)]),
    "cetra_periodic_search": (_INT, [_P, _P, _P, _INT, _P, _P, _P, _P, _P, _P,
                                     ctypes.POINTER(_I64)]),
    "cetra_mask_transits_device": (_INT, [_P, _P, _P, _SZ, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _P]),
    "cetra_mask_transits": (_INT, [_P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(_I64)]),
    "cetra_monotransit_workspace_bytes": (_SZ, [_P, _INT]),
    "cetra_monotransits_device": (_INT, [_P, _P, _P, _SZ, _INT, _P, _P]),
    "cetra_monotransit_search": (_INT, [_P, _P, _INT, _P, ctypes.POINTER(_INT)]),
    "cetra_search_iterative": (_INT, [_P, _P, _P, _INT, _P, _INT, ctypes.c_double, _P,
                                      ctypes.POINTER(_INT)]),
    "cetra_selftest_wait_timeout": (_INT, [_P, ctypes.POINTER(_INT), ctypes.POINTER(ctypes.c_double)]),
    "cetra_measure_peaks": (_INT, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "cetra_grid_free": (None, [_P]),
    "cetra_batch_create": (_INT, [_P, ctypes.POINTER(cetra_params), _INT, _P, _P, _P, _P, _P,
                                  _INT, _P, _INT, _P, _P, _P, _INT, ctypes.POINTER(_P)]),
    "cetra_batch_run": (_INT, [_P, _P, _P]),
    "cetra_batch_get_info": (_INT, [_P, ctypes.POINTER(cetra_batch_info)]),
    "cetra_batch_destroy": (None, [_P]),
    "cetra_batch_features": (_INT, [_P, _P, _INT, _P]),
    "cetra_batch_run_items": (_INT, [_P, _P, _P, _I64, _INT, _P]),
    "cetra_batch_curve": (_INT, [_P, _INT, _P, _P, _P, _P, _P, _P]),
    "cetra_cnn_create": (_INT, [_P, _INT, _INT, _INT, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "cetra_cnn_destroy": (None, [_P]),
    "cetra_cnn_param_count": (_I64, [_P]),
    "cetra_cnn_get_params": (_INT, [_P, _P, _P]),
    "cetra_cnn_set_params": (_INT, [_P, _P, _P]),
    "cetra_cnn_forward": (_INT, [_P, _P, _P, _INT, _P]),
    "cetra_cnn_backward": (_INT, [_P, _P, _P, _P, _INT, ctypes.c_float,
                                  ctypes.POINTER(ctypes.c_double), _P]),
    "cetra_cnn_adam": (_INT, [_P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float]),
    "cetra_batch_run_proposed": (_INT, [_P, _P, _P, _INT, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, _INT, _P, _P, _P, _P]),
    "cetra_cnn_map": (_INT, [_P, _P, _P, _INT, _INT, _INT, _P]),
    "cetra_cnn_shape": (_INT, [_P, ctypes.POINTER(_INT), ctypes.POINTER(_INT), ctypes.POINTER(_INT)]),
    "cetra_batch_search_proposed": (_INT, [_P, _P, _P, _INT, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, _P, _P, _P]),
    "cetra_cnn_comb": (_INT, [_P, _P, _INT, _INT, _P, _P, ctypes.c_double, ctypes.c_double, _INT,
                              _P]),
    "cetra_search_batch": (_INT, [_P, ctypes.POINTER(cetra_params), _INT, _P, _P, _P, _P, _P,
                                  _INT, _P, _INT, _P, _P, _P, _P]),
    "cetra_grid_get_info": (_INT, [_P, ctypes.POINTER(cetra_plan_info)]),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libcetra.so not built ({path}); run paper_2503_20875_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


def check(status: int, ctx=None, what: str = "") -> None:
    if status != CETRA_OK:
        msg = lib.cetra_last_error(ctx).decode() if ctx else ""
        raise CetraError(status, f"{what}: {msg}" if what else msg)


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(lib, name)
    raise AttributeError(name)
