"""The seeded input recipes and the roofline's work count, on CPU.

Each synthetic workload has the sampling, noise, injected planets and search grids its
description states (the shapes of the paper's TESS and Kepler use cases, Sec. 3 and Sec. 4),
and bench.py's algorithmic cell-read count of the fold (the numerator of its roofline,
Sec. 2.3: every (period, duration D < P, phase, epoch) cell inside the t0 grid) equals a
brute-force count.
"""
import math
import os
import sys

import numpy as np
import pytest

import synth
from synth.lightcurves import DAY_S, HOUR, inject_transits

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _noise(w):
    """flux minus the injected model: the noise the generator added."""
    return w.flux.astype(np.float64) - (1.0 - inject_transits(w.time, w.planets))


def _log_spaced(x, lo, hi, n):
    r = x[1:] / x[:-1]
    return (x.size == n and x[0] == pytest.approx(lo, rel=1e-12)
            and x[-1] == pytest.approx(hi, rel=1e-12) and np.allclose(r, r[0], rtol=1e-9))


def test_tess_2min_recipe():
    w = synth.make_workload("tess_2min_27d", seed=1)
    assert w.time.size == 19440
    assert np.allclose(np.diff(w.time), 120.0 / DAY_S, rtol=1e-9)
    assert w.t0_step == pytest.approx(120.0 / DAY_S) and w.cadence == pytest.approx(120.0 / DAY_S)
    assert _log_spaced(w.durations, 0.5 * HOUR, 6.0 * HOUR, 10)
    assert _log_spaced(w.periods, 0.5, 13.5, 2000)
    assert np.all(w.flux_err == np.float32(1000e-6))
    n = _noise(w)
    assert n.std() == pytest.approx(1000e-6, rel=0.03) and abs(n.mean()) < 5 * 1000e-6 / math.sqrt(n.size)
    (pl,) = w.planets
    assert (pl["P"], pl["depth"], pl["D"], pl["u1"], pl["u2"]) == (3.7, 1500e-6, 2.5 * HOUR, 0.4, 0.25)
    assert 0.0 <= pl["t0"] < 3.7
    d = inject_transits(w.time, w.planets)
    assert 0.97 * 1500e-6 < d.max() <= 1500e-6 * (1 + 1e-9)   # the deepest point is the depth
    assert np.count_nonzero(d) == pytest.approx(7 * 75, abs=8)  # ~7 transits of 75 points


def test_tess_20s_recipe():
    w = synth.make_workload("tess_20s_27d", seed=1)
    assert w.time.size == 116640 - 4320                        # minus the 1-d gap
    assert not np.any((w.time >= 13.0) & (w.time < 14.0))
    assert w.t0_step == pytest.approx(20.0 / DAY_S)
    assert _log_spaced(w.durations, 0.5 * HOUR, 12.0 * HOUR, 20)
    assert _log_spaced(w.periods, 0.5, 13.5, 50000)
    assert np.all(w.flux_err == np.float32(600e-6))
    n = _noise(w)
    # white 600 ppm plus stationary AR(1) of std 200 ppm and phi = 0.98
    assert n.std() == pytest.approx(math.hypot(600e-6, 200e-6), rel=0.03)
    seg = n[w.time < 13.0]                                     # contiguous samples only
    lag1 = np.corrcoef(seg[:-1], seg[1:])[0, 1]
    assert lag1 == pytest.approx(0.98 * 200e-6 ** 2 / (600e-6 ** 2 + 200e-6 ** 2), abs=0.02)
    got = sorted((p["depth"], p["P"]) for p in w.planets)
    assert got == [(300e-6, 5.1), (800e-6, 11.3)]
    for p in w.planets:
        assert p["D"] == pytest.approx(13.0 * HOUR * (p["P"] / 365.0) ** (1.0 / 3.0))


def test_kepler_4yr_recipe():
    w = synth.make_workload("kepler_1min_4yr", seed=1)
    assert w.time.size == 1461 * 1440
    assert w.time[0] == 2.45e6 and w.time[-1] - w.time[0] == pytest.approx(1461 - 1 / 1440)
    assert w.t0_step == pytest.approx(60.0 / DAY_S)
    assert _log_spaced(w.durations, 1.0 * HOUR, 16.0 * HOUR, 30)
    assert _log_spaced(w.periods, 1.0, 700.0, 100000)
    assert np.all(w.flux_err == np.float32(300e-6))
    assert _noise(w).std() == pytest.approx(300e-6, rel=0.03)
    (pl,) = w.planets
    assert (pl["P"], pl["depth"], pl["D"]) == (365.0, 90e-6, 13.0 * HOUR)
    assert np.count_nonzero(inject_transits(w.time, w.planets)) == pytest.approx(4 * 780, abs=8)


def test_batch_recipe():
    ws = synth.make_batch_workload(n_curves=256, seed=1)
    cad = 1800.0 / DAY_S
    sizes = np.array([w.time.size for w in ws])
    assert np.all(sizes % 1315 == 0) and sizes.min() >= 1315 and sizes.max() <= 13 * 1315
    assert len(set(sizes // 1315)) >= 10                       # sectors ~ U{1..13}
    n_planets = 0
    for w in ws:
        gaps = np.diff(w.time)
        assert np.all((np.abs(gaps - cad) < 1e-9) | (gaps > 1.0))  # 30-min cadence, 1-d gaps
        assert np.all(np.diff(np.flatnonzero(gaps > 1.0)) == 1315)
        T = w.time[-1] - w.time[0]
        # sigma_c exp(0.2 N(0, 1)) with sigma_c log-uniform in 500-5,000 ppm
        ls = np.log(w.flux_err.astype(np.float64))
        assert ls.std() == pytest.approx(0.2, rel=0.15)
        sig_c = math.exp(ls.mean())
        assert 500e-6 * 0.97 < sig_c < 5000e-6 * 1.03
        assert _log_spaced(w.durations, 1.0 * HOUR, 16.0 * HOUR, 16)
        ratio = 1.0 + w.durations[0] / (2.0 * T)
        assert w.periods[0] == 0.5 and w.periods[-1] <= T / 2.0 < w.periods[-1] * ratio * (1 + 1e-12)
        assert np.allclose(w.periods[1:] / w.periods[:-1], ratio, rtol=1e-9)
        for p in w.planets:
            n_planets += 1
            assert 1.0 <= p["P"] <= min(100.0, T / 2.0)
            n_in = max(1.0, (T / p["P"]) * p["D"] / cad)
            snr = p["depth"] * math.sqrt(n_in) / sig_c
            assert 5.0 * 0.95 < snr < 20.0 * 1.05
    assert 0.2 < n_planets / len(ws) < 0.4                     # 30 % carry a planet


@pytest.mark.parametrize("p,q", [(1, 1), (3, 2), (1, 4)])
def test_fold_cell_count_brute_force(p, q):
    sys.path.insert(0, ROOT)
    import bench
    c, I = 0.01, 157
    info = {"n_t0": I, "p": p, "q": q, "cadence": c}
    durations = np.array([0.02, 0.05, 0.3])
    periods = np.array([0.004, 0.01, 0.013, 0.1, 0.37, 0.5, 1.0, 1.57, 5.0])
    brute = 0
    for P in periods:
        Ps = (P * q) / (c * p)                                 # period in t0 steps
        if Ps < 1.0:
            continue                                           # no distinct phase: null
        nph = min(I, math.ceil(Ps))
        for D in durations:
            if not D < P:
                continue
            for i in range(nph):
                e = 0
                while i + math.floor(e * Ps + 0.5) < I:
                    brute += 1
                    e += 1
    assert bench.fold_cells(info, durations, periods) == brute
