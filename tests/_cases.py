"""Small hand-built inputs shared by the CPU pin tests and the GPU parity tests.

Nothing here computes any part of the search; it only lays out times, fluxes
and errors with known structure. Cadences are powers of two in days
(c = 2^-6 d = 22.5 min) so that tick arithmetic is exact and every window
edge used by a pin lies unambiguously inside or outside a window.
"""
import numpy as np

C_EXACT = 2.0 ** -6  # days


def regular(n, c=C_EXACT, t_start=0.0):
    return t_start + np.arange(n, dtype=np.float64) * c


def sigmas(rng, n, lo=0.5e-3, hi=2e-3):
    return rng.uniform(lo, hi, n).astype(np.float32)


def box_template(n=2):
    return np.ones(n, np.float32)
