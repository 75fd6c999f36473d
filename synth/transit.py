"""Quadratic limb-darkened transit profiles by numerical integration over the stellar disk.

Stellar intensity (quadratic law), mu = sqrt(1 - r^2):
    I(r) = 1 - u1 (1 - mu) - u2 (1 - mu)^2
Total flux:  F = int_0^1 I(r) 2 pi r dr = pi (1 - u1/3 - u2/6).
A planet of radius p (stellar radii) at projected separation z hides, on the
stellar annulus of radius r, the arc of half-angle
    kappa(r) = pi                                   if r <= p - z
             = arccos((r^2 + z^2 - p^2) / (2 r z))  if |z - p| < r < z + p
             = 0                                    otherwise,
so the fractional deficit is  delta(z) = int_0^1 I(r) 2 r kappa(r) dr / F.
"""
from __future__ import annotations

import functools

import numpy as np


def ld_deficit(z, p, u1, u2, n_r=2048):
    """Fractional flux deficit delta(z) for each separation in ``z`` (midpoint rule in r)."""
    z = np.atleast_1d(np.asarray(z, np.float64))
    out = np.zeros_like(z)
    F = np.pi * (1.0 - u1 / 3.0 - u2 / 6.0)
    for k, zk in enumerate(z):
        r_lo = max(0.0, zk - p)
        r_hi = min(1.0, zk + p)
        if r_hi <= r_lo:
            continue
        h = (r_hi - r_lo) / n_r
        r = r_lo + (np.arange(n_r) + 0.5) * h
        mu = np.sqrt(np.clip(1.0 - r * r, 0.0, 1.0))
        inten = 1.0 - u1 * (1.0 - mu) - u2 * (1.0 - mu) ** 2
        if zk == 0.0:
            kap = np.where(r <= p, np.pi, 0.0)
        else:
            cosk = (r * r + zk * zk - p * p) / (2.0 * r * zk)
            kap = np.arccos(np.clip(cosk, -1.0, 1.0))
            kap = np.where(r <= p - zk, np.pi, kap)
        out[k] = np.sum(inten * 2.0 * r * kap) * h / F
    return out


@functools.lru_cache(maxsize=64)
def _profile(n_samples, b, p, u1, u2):
    X = np.sqrt((1.0 + p) ** 2 - b * b)
    x = np.arange(n_samples, dtype=np.float64) / (n_samples - 1)
    z = np.sqrt(b * b + (X * (2.0 * x - 1.0)) ** 2)
    prof = ld_deficit(z, p, u1, u2)
    prof[0] = 0.0
    prof[-1] = 0.0
    prof.setflags(write=False)
    return prof


def ld_transit_template(n_samples=4096, b=0.32, p=0.03, u1=0.4804, u2=0.1867, normalise=True):
    """Transit deficit sampled at x = k/(n-1), x = 0 first contact, x = 1 last contact.

    The planet crosses on a straight chord at impact parameter b; between the
    contacts the projected separation is z(x) = sqrt(b^2 + (X (2x - 1))^2),
    X = sqrt((1 + p)^2 - b^2).
    """
    if b >= 1.0 + p:
        raise ValueError("impact parameter gives no transit")
    prof = _profile(int(n_samples), float(b), float(p), float(u1), float(u2)).copy()
    if normalise:
        prof = prof / prof.max()
    return prof


_DEFAULT = None


def default_template(n_samples=4096):
    """The paper's default model (Sec. 2.1.2): Rp = 0.03 R*, b = 0.32, u1, u2 = 0.4804, 0.1867."""
    global _DEFAULT
    if _DEFAULT is None or _DEFAULT.size != n_samples:
        _DEFAULT = ld_transit_template(n_samples, b=0.32, p=0.03, u1=0.4804, u2=0.1867)
    return _DEFAULT.copy()
