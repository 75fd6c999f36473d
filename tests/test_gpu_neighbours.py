"""Method neighbours on the GPU against the oracle: masking a detected signal and the
iterative search (Sec. 4.2, reading R17), single-transit events (Sec. 1, Sec. 5, reading R18)."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from synth.lightcurves import HOUR
from tests._parity import compare_linear, oracle_search

pytestmark = pytest.mark.gpu

CAD = 1.0 / 64.0


def _curve(n=64 * 30, planets=(), sigma=1e-3, seed=1, durations_h=(2.0, 4.0, 8.0)):
    t = np.arange(n, dtype=np.float64) * CAD
    rng = np.random.default_rng(seed)
    f = 1.0 - synth.inject_transits(t, list(planets)) + rng.normal(0.0, sigma, n)
    return t, f.astype(np.float32), np.full(n, sigma, np.float32), np.array(durations_h) * HOUR


def _device(ctx, t, f, e, d, workspace_bytes=None, **params):
    import torch
    from paper_2503_20875_gb300 import Plan
    plan = Plan(ctx, t, f, e, d, synth.default_template(1024), **params)
    nb = workspace_bytes(plan) if workspace_bytes else plan.workspace_bytes(0)
    ws = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    dt = torch.as_tensor(t, device="cuda")
    df = torch.as_tensor(f, device="cuda")
    de = torch.as_tensor(e, device="cuda")
    return plan, ws, (dt, df, de)


def test_mask_then_linear_matches_oracle():
    """Dyadic times, period, mid-time and half-width (exact arithmetic, cells exactly h away
    kept): the same cells are nulled, and the linear search of the masked curve matches the
    oracle's element by element, null cells included."""
    import torch
    from paper_2503_20875_gb300 import (Context, cetra_resample_device, cetra_linear_device,
                                        cetra_mask_transits_device)
    pl = [dict(P=4.0, t0=1.5, D=3 * HOUR, depth=2e-3)]
    t, f, e, d = _curve(planets=pl)
    ctx = Context(0)
    plan, ws, (dt, df, de) = _device(ctx, t, f, e, d, cadence=CAD, t0_step=CAD)
    cetra_resample_device(ctx, plan, dt, df, de, ws)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    cetra_mask_transits_device(ctx, plan, ws, 4.0, 1.5, 0.125, cnt)
    J, I = d.size, plan.info["n_t0"]
    out = {k: torch.empty((J, I), dtype=torch.float32, device="cuda")
           for k in ("depth", "depth_var", "dlogl")}
    cetra_linear_device(ctx, plan, ws, out["depth"], out["depth_var"], out["dlogl"])
    torch.cuda.synchronize()
    g = oracle.geometry(t, f, e, d, cadence=CAD, t0_step=CAD)
    y, w = oracle.resample(t, f, e, g)
    y2, w2, n = oracle.mask_transits(g, y, w, 4.0, 1.5, 0.125)
    assert int(cnt.item()) == n and n > 0
    T = oracle.template(synth.default_template(1024), 1024)
    dep, var, lr, kap = oracle.linear(g, y2, w2, d, T, with_kappa=True)
    gpu = {k: v.cpu().numpy() for k, v in out.items()}
    compare_linear(gpu, {"depth": dep, "depth_var": var, "dlogl": lr, "kappa": kap, "geom": g}, d)
    # half_width 0 masks nothing
    cetra_mask_transits_device(ctx, plan, ws, 4.0, 1.5, 0.0, cnt)


def test_iterative_search_matches_oracle():
    """Three rounds of search-and-mask on a curve with two planets: every round's best
    (period index, t0, duration) equals the oracle's, LR within 1e-5."""
    from paper_2503_20875_gb300 import Context, cetra_linear_search, cetra_search_iterative
    pl = [dict(P=3.3, t0=0.7, D=3 * HOUR, depth=3e-3), dict(P=5.7, t0=2.1, D=3 * HOUR, depth=2e-3)]
    t, f, e, d = _curve(planets=pl, seed=3, durations_h=(2.0, 3.0, 4.0))
    periods = np.exp(np.linspace(np.log(1.0), np.log(12.0), 600))
    tm = synth.default_template(1024)
    ref, _ = oracle.search_iterative(t, f, e, d, tm, periods, 3, cadence=CAD, t0_step=CAD)
    ctx = Context(0)
    grid, _, _, _ = cetra_linear_search(ctx, t, f, e, d, tm, outputs=False, cadence=CAD,
                                        t0_step=CAD)
    got = cetra_search_iterative(ctx, grid, periods, n_iter=3, width=2.0)
    assert len(got["k"]) == len(ref) == 3
    for r, det in enumerate(ref):
        assert got["k"][r] == det["k"]
        assert got["t0"][r] == det["t0"]
        assert got["duration"][r] == det["duration"]
        assert got["j"][r] == det["j"]
        assert got["dlogl"][r] == pytest.approx(det["dlogl"], rel=1e-5)
        assert got["depth"][r] == pytest.approx(det["depth"], rel=1e-5)
    assert abs(got["period"][0] - 3.3) < 0.033 and abs(got["period"][1] - 5.7) < 0.057
    # argument errors are refused before any launch
    from paper_2503_20875_gb300 import CetraError, cetra_mask_transits
    for bad in ((0.0, 1.0, 0.1), (float("nan"), 1.0, 0.1), (2.0, float("inf"), 0.1),
                (2.0, 1.0, -0.1)):
        with pytest.raises(CetraError):
            cetra_mask_transits(ctx, grid, *bad)
    with pytest.raises(CetraError):
        cetra_search_iterative(ctx, grid, periods, n_iter=0)


def _compare_events(got_i, got_j, got_lr, g, d, dep, lr, n_ref_i, n_ref_j):
    """Events equal the oracle's in order; a mismatch is allowed only as an epsilon-tie (the
    oracle's LR at the GPU's window within 1e-5 of the oracle's pick), after which later
    events may legitimately differ."""
    assert len(got_i) == len(n_ref_i)
    for m, (gi, gj, ri, rj) in enumerate(zip(got_i, got_j, n_ref_i, n_ref_j)):
        if (gi, gj) != (ri, rj):
            assert lr[rj, ri] - lr[gj, gi] <= 1e-5 * lr[rj, ri], (m, gi, gj, ri, rj)
            return m
        assert got_lr[m] == pytest.approx(lr[rj, ri], rel=1e-5)
    return len(got_i)


def test_monotransits_match_oracle():
    """Host and device paths against the oracle on single transits plus noise."""
    import torch
    from paper_2503_20875_gb300 import (Context, cetra_linear_search, cetra_monotransit_search,
                                        cetra_resample_device, cetra_linear_device,
                                        cetra_monotransits_device)
    from paper_2503_20875_gb300 import _native as N
    pl = [dict(P=np.inf, t0=t0, D=4 * HOUR, depth=dep)
          for t0, dep in ((4.0, 2e-3), (11.0, 4e-3), (19.5, 3e-3), (25.2, 1.2e-3))]
    t, f, e, d = _curve(planets=pl, sigma=5e-4, durations_h=(2.0, 4.0, 8.0))
    tm = synth.default_template(1024)
    r = oracle.search(t, f, e, d, tm, cadence=CAD, t0_step=CAD / 4)
    g = r["geom"]
    ri, rj = oracle.monotransits(g, d, r["depth"], r["dlogl"], 12)
    ctx = Context(0)
    grid, _, _, _ = cetra_linear_search(ctx, t, f, e, d, tm, outputs=False, cadence=CAD,
                                        t0_step=CAD / 4)
    ev = cetra_monotransit_search(ctx, grid, 12)
    n_same = _compare_events(ev["i"], ev["j"], ev["dlogl"], g, d, r["depth"], r["dlogl"], ri, rj)
    assert n_same >= 4
    for m in range(n_same):
        assert ev["t0"][m] == oracle.t0_of(g, ri[m])
        assert ev["duration"][m] == d[rj[m]]
        assert ev["depth"][m] == pytest.approx(r["depth"][rj[m], ri[m]], rel=1e-5)
    # the three strongest injected transits come first, strongest first; the weakest is
    # found too (a window just outside the deepest event's duration, straddling its edge,
    # may rank before it)
    for m, t0 in enumerate((11.0, 19.5, 4.0)):
        assert abs(ev["t0"][m] - t0) <= 2 * g.t0_step
    assert np.min(np.abs(ev["t0"] - 25.2)) <= 2 * g.t0_step
    # device path: the same events
    plan, ws, (dt, df, de) = _device(
        ctx, t, f, e, d, workspace_bytes=lambda p: N.lib.cetra_monotransit_workspace_bytes(p.handle, 12),
        cadence=CAD, t0_step=CAD / 4)
    cetra_resample_device(ctx, plan, dt, df, de, ws)
    cetra_linear_device(ctx, plan, ws, None, None, None)
    rec = ctypes.sizeof(N.cetra_event)
    d_ev = torch.zeros(12 * rec, dtype=torch.uint8, device="cuda")
    d_n = torch.zeros(1, dtype=torch.int32, device="cuda")
    cetra_monotransits_device(ctx, plan, ws, 12, d_ev, d_n)
    torch.cuda.synchronize()
    n = int(d_n.item())
    raw = d_ev.cpu().numpy().tobytes()
    dev_ev = [N.cetra_event.from_buffer_copy(raw[rec * m:rec * (m + 1)]) for m in range(n)]
    assert n == len(ev["i"])
    assert [x.i for x in dev_ev] == list(ev["i"]) and [x.j for x in dev_ev] == list(ev["j"])


def test_monotransits_tess_2min_and_limits():
    """A whole 27-d 2-min curve (periodic planet: its transits are the strongest events) and
    the argument limits."""
    from paper_2503_20875_gb300 import Context, CetraError, cetra_linear_search, cetra_monotransit_search
    w = synth.make_workload("tess_2min_27d")
    r = oracle.search(w.time, w.flux, w.flux_err, w.durations, w.template, cadence=w.cadence,
                      t0_step=w.t0_step)
    g = r["geom"]
    ri, rj = oracle.monotransits(g, w.durations, r["depth"], r["dlogl"], 10)
    ctx = Context(0)
    grid, _, _, _ = cetra_linear_search(ctx, w.time, w.flux, w.flux_err, w.durations, w.template,
                                        outputs=False, cadence=w.cadence, t0_step=w.t0_step)
    ev = cetra_monotransit_search(ctx, grid, 10)
    n_same = _compare_events(ev["i"], ev["j"], ev["dlogl"], g, w.durations, r["depth"],
                             r["dlogl"], ri, rj)
    assert n_same >= 3
    P, t0 = w.planets[0]["P"], w.planets[0]["t0"]
    ph = (ev["t0"][:3] - t0 + 0.5 * P) % P - 0.5 * P
    assert np.all(np.abs(ph) < 0.1)
    with pytest.raises(CetraError):
        cetra_monotransit_search(ctx, grid, 0)
    with pytest.raises(CetraError):
        cetra_monotransit_search(ctx, grid, 5000)
