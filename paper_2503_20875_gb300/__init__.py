"""GB300-native (sm_103a) CETRA transit search: linear search + periodic search.

The compute lives in ``libcetra.so`` (CUDA kernels behind the C ABI of
include/cetra.h), built in-tree by ``paper_2503_20875_gb300.build.build()``.
Importing this package loads that library and fails loudly if it is absent.
"""
from .api import (Context, Plan, DeviceSearch, LinearGrid, Batch, make_params,
                  cetra_linear_search, cetra_periodic_search, cetra_resample_device,
                  cetra_linear_device, cetra_periodic_device, cetra_logl0_device,
                  cetra_search_batch, CNN, cetra_cnn_map, cetra_cnn_comb,
                  cetra_mask_transits, cetra_monotransit_search, cetra_search_iterative,
                  cetra_mask_transits_device, cetra_monotransits_device,
                  cetra_selftest_wait_timeout, cetra_measure_peaks)
from ._native import CetraError, LIB_PATH

__all__ = ["Context", "Plan", "DeviceSearch", "LinearGrid", "Batch", "cetra_search_batch",
           "CNN", "cetra_cnn_map", "cetra_cnn_comb", "cetra_mask_transits",
           "cetra_monotransit_search", "cetra_search_iterative", "cetra_mask_transits_device",
           "cetra_monotransits_device", "cetra_selftest_wait_timeout", "cetra_measure_peaks",
           "make_params", "cetra_linear_search",
           "cetra_periodic_search", "cetra_resample_device", "cetra_linear_device",
           "cetra_periodic_device", "cetra_logl0_device", "CetraError", "LIB_PATH"]
