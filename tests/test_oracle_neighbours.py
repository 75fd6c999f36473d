"""Pins of the oracle's method-neighbour steps: masking a detected signal (Sec. 4.2, reading
R17) and single-transit events from the linear search (Sec. 1, Sec. 5, reading R18)."""
from fractions import Fraction
import math

import numpy as np
import pytest

import oracle
import synth
from synth.lightcurves import HOUR

CAD = 1.0 / 64.0  # 22.5 min: a dyadic cadence keeps the mask arithmetic exact


def _curve(n=64 * 30, planets=(), sigma=1e-3, seed=1, durations_h=(2.0, 4.0, 8.0), noise=True):
    t = np.arange(n, dtype=np.float64) * CAD
    rng = np.random.default_rng(seed)
    f = 1.0 - synth.inject_transits(t, list(planets))
    if noise:
        f = f + rng.normal(0.0, sigma, n)
    return t, f.astype(np.float32), np.full(n, sigma, np.float32), np.array(durations_h) * HOUR


def test_mask_cells_exact():
    """Dyadic t, P, t0 and half-width: the nulled cells are exactly those within h of a
    mid-time, computed in rational arithmetic; cells exactly h away are kept."""
    t, f, e, d = _curve()
    g = oracle.geometry(t, f, e, d, cadence=CAD, t0_step=CAD)
    y, w = oracle.resample(t, f, e, g)
    P, t0, h = 4.0, 1.5, 0.125
    y2, w2, n = oracle.mask_transits(g, y, w, P, t0, h)
    want = set()
    for k in range(g.n_grid):
        gk = Fraction(k - g.n_pad, 64)
        dd = gk - Fraction(3, 2)
        m = math.floor(dd / 4 + Fraction(1, 2))
        if abs(dd - 4 * m) < Fraction(1, 8):
            want.add(k)
    got = set(np.nonzero((w2 == 0) & (w > 0))[0].tolist())
    assert got == {k for k in want if w[k] > 0}
    assert n == len(got)
    assert np.all(w2[sorted(want)] == 0) and np.all(y2[sorted(want)] == 0)
    keep = np.setdiff1d(np.arange(g.n_grid), sorted(want))
    np.testing.assert_array_equal(w2[keep], w[keep])
    np.testing.assert_array_equal(y2[keep], y[keep])
    # boundary cells (exactly h from a mid-time) exist and are kept
    edge = [k for k in range(g.n_grid)
            if abs((Fraction(k - g.n_pad, 64) - Fraction(3, 2)) % 4 - 2) == 2 - Fraction(1, 8)]
    assert edge and not set(edge) & want
    # masking the same signal again nulls nothing new
    _, w3, n3 = oracle.mask_transits(g, y2, w2, P, t0, h)
    assert n3 == 0 and np.array_equal(w3, w2)


def test_iterative_search_finds_both_planets():
    """Two planets: the first search finds the stronger one; after masking it, the second
    search finds the other (periods within 1 %, Sec. 3.1)."""
    pl = [dict(P=3.3, t0=0.7, D=3 * HOUR, depth=3e-3), dict(P=5.7, t0=2.1, D=3 * HOUR, depth=2e-3)]
    t, f, e, d = _curve(planets=pl, sigma=1e-3, seed=3, durations_h=(2.0, 3.0, 4.0))
    periods = np.exp(np.linspace(np.log(1.0), np.log(12.0), 600))
    dets, g = oracle.search_iterative(t, f, e, d, synth.default_template(1024), periods, 3,
                                      cadence=CAD, t0_step=CAD)
    assert len(dets) == 3
    assert abs(dets[0]["period"] - 3.3) <= 0.033
    assert abs(dets[1]["period"] - 5.7) <= 0.057
    assert dets[1]["depth"] == pytest.approx(2e-3, rel=0.3)
    # the third search sees neither planet (nor a harmonic of one) any more, and is weaker
    for Pt in (3.3, 5.7):
        assert all(abs(dets[2]["period"] - m * Pt) > 0.01 * m * Pt for m in (0.5, 1.0, 2.0))
    assert dets[2]["dlogl"] < 0.5 * dets[1]["dlogl"]


def _sort_and_scan(g, durations, depth, lr, max_events):
    """The greedy events as one pass over the windows sorted by (-LR, j, i): accept a
    window unless an accepted event hides it."""
    J, I = lr.shape
    cand = [(-lr[j, i], j, i) for j in range(J) for i in range(I)
            if not np.isnan(lr[j, i]) and depth[j, i] > 0]
    cand.sort()
    out = []
    for _, j, i in cand:
        if len(out) == max_events:
            break
        if any(float(abs(i - ie)) < (durations[je] * g.q) / (g.cadence * g.p) for ie, je in out):
            continue
        out.append((i, j))
    return out


@pytest.mark.parametrize("seed,durations_h,step", [
    (0, (1.0, 2.5, 5.0), CAD / 2), (1, (1.0, 2.5, 5.0), CAD / 2), (2, (1.0, 2.5, 5.0), CAD / 2),
    # durations of exactly 2, 4 and 8 t0 steps: cells exactly one duration away stay visible
    (3, (0.75, 1.5, 3.0), CAD), (4, (0.75, 1.5, 3.0), CAD)])
def test_monotransits_equal_sort_and_scan(seed, durations_h, step):
    t, f, e, d = _curve(n=600, durations_h=durations_h)
    g = oracle.geometry(t, f, e, d, cadence=CAD, t0_step=step)
    rng = np.random.default_rng(seed)
    J, I = d.size, g.n_t0
    lr = np.round(rng.exponential(3.0, size=(J, I)), 1)  # rounding makes exact ties
    depth = rng.normal(size=(J, I))
    lr[rng.uniform(size=(J, I)) < 0.05] = np.nan
    ii, jj = oracle.monotransits(g, d, depth, lr, 12)
    assert list(zip(ii.tolist(), jj.tolist())) == _sort_and_scan(g, d, depth, lr, 12)
    # no eligible window: nothing
    ii, _ = oracle.monotransits(g, d, -np.abs(depth), lr, 5)
    assert ii.size == 0


def test_monotransits_recover_injected_single_transits():
    """Three single transits (no period) of different depths, low noise: the three
    strongest events are those transits, strongest first, at the injected mid-times
    (within one t0 step) and durations."""
    pl = [dict(P=np.inf, t0=t0, D=4 * HOUR, depth=dep)
          for t0, dep in ((4.0, 2e-3), (11.0, 4e-3), (19.5, 3e-3))]
    t, f, e, d = _curve(planets=pl, sigma=2e-4, durations_h=(2.0, 4.0, 8.0))
    r = oracle.search(t, f, e, d, synth.default_template(1024), cadence=CAD, t0_step=CAD)
    g = r["geom"]
    ii, jj = oracle.monotransits(g, d, r["depth"], r["dlogl"], 3)
    assert ii.size == 3
    for (i, j), t0 in zip(zip(ii, jj), (11.0, 19.5, 4.0)):
        assert abs(oracle.t0_of(g, i) - t0) <= g.t0_step
        assert j == 1
