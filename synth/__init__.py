"""Seeded synthetic inputs for the CETRA search: transit templates and light curves.

This module serves both the CUDA path and the FP64 oracle and holds none of the
search's arithmetic (no resampling, windowing or folding). It draws every
random number with numpy's PCG64 from an explicit seed.

Contents
  ld_transit_template  quadratic limb-darkened transit profile, first to last
                       contact, max-normalised, by numerical integration over
                       the stellar disk (written from first principles).
  default_template     the paper's default model parameters (Sec. 2.1.2:
                       Rp = 0.03 R*, b = 0.32, u1, u2 = 0.4804, 0.1867).
  log_grid             log-spaced duration / period grids.
  WORKLOADS            the synthetic stand-ins for the five workload shapes
                       (single TESS-like curves, a high-cadence curve, a
                       multi-year Kepler/PLATO-like curve, a batch of uneven
                       curves), built by make_workload(name, seed).
"""
from .transit import ld_transit_template, default_template, ld_deficit
from .lightcurves import (log_grid, inject_transits, make_workload, WORKLOADS, Workload,
                          make_batch_workload, make_batch_csr)

__all__ = ["ld_transit_template", "default_template", "ld_deficit", "log_grid",
           "inject_transits", "make_workload", "WORKLOADS", "Workload", "make_batch_workload", "make_batch_csr"]
