"""Seeded synthetic light curves shaped like TESS, Kepler and PLATO photometry.

Each workload fixes the time sampling, the noise model, the injected planets
and the search grids (durations, t0 step, periods). The paper evaluates on
real TESS light curves and on 173-d synthetic curves (Sec. 3.1, Sec. 4); none
of those data are used here: these seeded curves stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .transit import ld_transit_template, default_template

DAY_S = 86400.0
HOUR = 1.0 / 24.0


def log_grid(lo, hi, n):
    """n values log-spaced from lo to hi inclusive (FP64)."""
    if n == 1:
        return np.array([lo], np.float64)
    return np.exp(np.linspace(np.log(lo), np.log(hi), int(n)))


@dataclass
class Workload:
    name: str
    time: np.ndarray          # float64 days (absolute)
    flux: np.ndarray          # float32, normalised to a baseline of 1
    flux_err: np.ndarray      # float32
    durations: np.ndarray     # float64 days
    periods: np.ndarray       # float64 days
    cadence: float            # resample cadence (days)
    t0_step: float            # t0 grid step (days)
    template: np.ndarray      # float32 dense template (first to last contact)
    planets: list = field(default_factory=list)
    description: str = ""


def inject_transits(time, planets, n_tmpl=2048):
    """Sum of the fractional deficits of ``planets`` at ``time``.

    Each planet: dict(P, t0 (mid-time), D, depth, b, u1, u2, rp). The shape is a
    limb-darkened profile from first to last contact scaled so its deepest
    point equals ``depth``.
    """
    deficit = np.zeros(time.size, np.float64)
    for pl in planets:
        prof = ld_transit_template(n_tmpl, b=pl.get("b", 0.32), p=pl.get("rp", 0.03),
                                   u1=pl.get("u1", 0.4804), u2=pl.get("u2", 0.1867))
        P, t0, D = pl["P"], pl["t0"], pl["D"]
        # phase of each point relative to the nearest transit centre
        ph = time - t0
        if np.isfinite(P):
            ph = ph - np.round(ph / P) * P
        x = (ph + 0.5 * D) / D
        inside = (x >= 0.0) & (x <= 1.0)
        xs = x[inside] * (n_tmpl - 1)
        deficit[inside] += pl["depth"] * np.interp(xs, np.arange(n_tmpl), prof)
    return deficit


def _ar1(rng, n, phi, std):
    """Stationary AR(1) with coefficient phi and marginal standard deviation std."""
    from scipy.signal import lfilter
    eps = rng.normal(0.0, std * np.sqrt(1.0 - phi * phi), n)
    x0 = rng.normal(0.0, std)
    out = lfilter([1.0], [1.0, -phi], eps, zi=np.array([phi * x0]))[0]
    return out


def _finish(name, t, deficit, noise, sigma, durations, periods, cadence, t0_step, planets, desc,
            rng=None, template_samples=4096):
    flux = (1.0 - deficit + noise).astype(np.float32)
    err = np.broadcast_to(np.asarray(sigma, np.float64), t.shape).astype(np.float32)
    return Workload(name, t, flux, err.copy(), np.asarray(durations, np.float64),
                    np.asarray(periods, np.float64), float(cadence), float(t0_step),
                    default_template(template_samples).astype(np.float32), planets, desc)


def tess_2min_27d(seed=1, n_periods=2000):
    """27 d at 2-min cadence (19,440 points), white noise 1000 ppm, one planet.

    Injected: quadratic LD (u1 = 0.4, u2 = 0.25), depth 1500 ppm, P = 3.7 d,
    D = 2.5 h, b = 0.3, t0 ~ U(0, P). Grids: 10 log-spaced durations 0.5-6 h,
    t0 step 2 min, 2,000 log-spaced periods 0.5-13.5 d.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cad = 120.0 / DAY_S
    t = np.arange(19440, dtype=np.float64) * cad
    planets = [dict(P=3.7, t0=float(rng.uniform(0.0, 3.7)), D=2.5 * HOUR, depth=1500e-6, b=0.3,
                    u1=0.4, u2=0.25, rp=0.03)]
    noise = rng.normal(0.0, 1000e-6, t.size)
    return _finish("tess_2min_27d", t, inject_transits(t, planets), noise, 1000e-6,
                   log_grid(0.5 * HOUR, 6.0 * HOUR, 10), log_grid(0.5, 13.5, n_periods), cad, cad,
                   planets, tess_2min_27d.__doc__)


def tess_20s_27d(seed=1, n_periods=50000):
    """27 d at 20-s cadence (116,640 samples) minus a 1-d gap (days 13-14), two planets.

    Noise: white 600 ppm plus AR(1) red noise (phi = 0.98, stationary std
    200 ppm); the error column is the white level, 600 ppm. Planets: 300 ppm at
    P = 5.1 d and 800 ppm at P = 11.3 d, D = 13 h (P / 365 d)^(1/3). Grids: 20
    log-spaced durations 0.5-12 h, t0 step 20 s, 50,000 log-spaced periods
    0.5-13.5 d.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cad = 20.0 / DAY_S
    t = np.arange(116640, dtype=np.float64) * cad
    t = t[(t < 13.0) | (t >= 14.0)]
    planets = []
    for depth, P in ((300e-6, 5.1), (800e-6, 11.3)):
        D = 13.0 * HOUR * (P / 365.0) ** (1.0 / 3.0)
        planets.append(dict(P=P, t0=float(rng.uniform(0.0, P)), D=D, depth=depth, b=0.3,
                            u1=0.4804, u2=0.1867, rp=0.03))
    noise = rng.normal(0.0, 600e-6, t.size) + _ar1(rng, t.size, 0.98, 200e-6)
    return _finish("tess_20s_27d", t, inject_transits(t, planets), noise, 600e-6,
                   log_grid(0.5 * HOUR, 12.0 * HOUR, 20), log_grid(0.5, 13.5, n_periods), cad, cad,
                   planets, tess_20s_27d.__doc__)


def kepler_1min_4yr(seed=1, n_periods=100000):
    """4-yr baseline (1461 d) at 1-min cadence (2,103,840 points), times offset by 2.45e6 d.

    White noise 300 ppm; an Earth analogue of depth 90 ppm, P = 365 d,
    D = 13 h. Grids: 30 log-spaced durations 1-16 h, t0 step 60 s, 100,000
    log-spaced periods 1-700 d.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cad = 60.0 / DAY_S
    n = 1461 * 1440
    t0_abs = 2.45e6
    t = t0_abs + np.arange(n, dtype=np.float64) * cad
    planets = [dict(P=365.0, t0=t0_abs + float(rng.uniform(0.0, 365.0)), D=13.0 * HOUR,
                    depth=90e-6, b=0.3, u1=0.4804, u2=0.1867, rp=0.03)]
    noise = rng.normal(0.0, 300e-6, n)
    return _finish("kepler_1min_4yr", t, inject_transits(t, planets), noise, 300e-6,
                   log_grid(1.0 * HOUR, 16.0 * HOUR, 30), log_grid(1.0, 700.0, n_periods), cad,
                   cad, planets, kepler_1min_4yr.__doc__)


def custom(seed=1, n_points=2000, cadence_s=120.0, sigma=1e-3, durations_h=(1.0, 2.0, 3.0),
           periods=None, t0_step_s=None, planets=None, gaps=(), jitter=0.0, sigma_spread=0.0,
           time_offset=0.0, drop_frac=0.0):
    """A small seeded curve for parity tests: optional gaps, jittered times,
    per-point sigma spread (lognormal), dropped points and time offset."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cad = cadence_s / DAY_S
    t = np.arange(n_points, dtype=np.float64) * cad
    if jitter:
        t = t + rng.uniform(-jitter, jitter, t.size) * cad
    for lo, hi in gaps:
        t = t[(t < lo) | (t >= hi)]
    if drop_frac:
        t = t[rng.uniform(size=t.size) >= drop_frac]
    sig = sigma * np.exp(sigma_spread * rng.normal(size=t.size))
    planets = list(planets or [])
    noise = rng.normal(size=t.size) * sig
    w = _finish("custom", t + time_offset, inject_transits(t, planets), noise, sig,
                np.asarray(durations_h, np.float64) * HOUR,
                np.asarray(periods if periods is not None else [1.0], np.float64), cad,
                (t0_step_s / DAY_S) if t0_step_s else cad, planets, custom.__doc__)
    return w


WORKLOADS = {
    "tess_2min_27d": tess_2min_27d,
    "tess_20s_27d": tess_20s_27d,
    "kepler_1min_4yr": kepler_1min_4yr,
}


def make_workload(name, seed=1, **kw):
    return WORKLOADS[name](seed=seed, **kw)


def make_batch_workload(n_curves=8192, seed=1, max_sectors=13, planet_frac=0.3,
                        snr_range=(5.0, 20.0), min_sectors=1, with_periods=True):
    """Batch of uneven 30-min curves: S ~ U{1..13} sectors of 27.4 d with 1-d gaps.

    Per-curve sigma_c log-uniform 500-5,000 ppm, per-point sigma = sigma_c
    exp(0.2 N(0, 1)); a fraction planet_frac (30 %) of curves carries one planet
    with P log-uniform in [1, min(100, T/2)] d and SNR ~ U(snr_range) (5-20),
    depth = SNR sigma_c / sqrt(n_in).
    Returns a list of Workload (16 log-spaced durations 1-16 h, t0 step 10 min,
    periods log-spaced from 0.5 d to T/2 with ratio 1 + D_min / (2 T); an empty period
    array when with_periods is False).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    cad = 1800.0 / DAY_S
    out = []
    durations = log_grid(1.0 * HOUR, 16.0 * HOUR, 16)
    for c in range(n_curves):
        S = int(rng.integers(min_sectors, max_sectors + 1))
        segs = []
        start = 0.0
        for _ in range(S):
            n_s = int(np.floor(27.4 / cad))
            segs.append(start + np.arange(n_s) * cad)
            start += 27.4 + 1.0
        t = np.concatenate(segs)
        T = t[-1] - t[0]
        sig_c = float(np.exp(rng.uniform(np.log(500e-6), np.log(5000e-6))))
        sig = sig_c * np.exp(0.2 * rng.normal(size=t.size))
        planets = []
        if rng.uniform() < planet_frac:
            P = float(np.exp(rng.uniform(np.log(1.0), np.log(min(100.0, T / 2.0)))))
            D = 13.0 * HOUR * (P / 365.0) ** (1.0 / 3.0)
            snr = float(rng.uniform(*snr_range))
            n_in = max(1.0, (T / P) * D / cad)
            planets.append(dict(P=P, t0=float(rng.uniform(0.0, P)), D=D,
                                depth=snr * sig_c / np.sqrt(n_in), b=0.3, u1=0.4804, u2=0.1867,
                                rp=0.03))
        noise = rng.normal(size=t.size) * sig
        ratio = 1.0 + durations[0] / (2.0 * T)
        n_p = int(np.floor(np.log((T / 2.0) / 0.5) / np.log(ratio))) + 1 if with_periods else 0
        periods = 0.5 * ratio ** np.arange(n_p)
        out.append(_finish(f"batch_{c}", t, inject_transits(t, planets), noise, sig, durations,
                           periods, cad, 600.0 / DAY_S, planets, "batch member"))
    return out


def make_batch_csr(job):
    """make_batch_workload packed back to back: job = (n_curves, seed, planet_frac).
    Returns (offsets int64 [n + 1], time f64, flux f32, flux_err f32, planets per curve);
    a top-level function so that process pools can call it."""
    n, seed, planet_frac = job
    ws = make_batch_workload(n_curves=n, seed=seed, planet_frac=planet_frac,
                             with_periods=False)
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum([w.time.size for w in ws])
    return (off, np.concatenate([w.time for w in ws]), np.concatenate([w.flux for w in ws]),
            np.concatenate([w.flux_err for w in ws]), [w.planets for w in ws])
