"""GPU parity: the CUDA path against the FP64 oracle, element by element, on
seeded inputs (tolerances in tests/_parity.py). Small cases span several
kernel tiles, ragged tails, chunked windows, every phase-class shape and the
degenerate cases; the full-size workloads run in the configuration the
benchmark times."""
import numpy as np
import pytest

import synth
from synth.lightcurves import custom, HOUR
from tests._cases import C_EXACT, regular, sigmas, box_template
from tests._parity import gpu_search, oracle_search, compare_linear, compare_periodic

pytestmark = pytest.mark.gpu


def _run_both(w, periods=None, mask=None, L=1024, **kw):
    args = (w.time, w.flux, w.flux_err, w.durations, w.template)
    prm = dict(cadence=kw.get("cadence", w.cadence), t0_step=kw.get("t0_step", w.t0_step),
               flux_is_offset=kw.get("flux_is_offset", False))
    P = w.periods if periods is None else periods
    g = gpu_search(*args, P, mask, L=L, **prm)
    o = oracle_search(*args, P, mask, L=L, **prm)
    return g, o


def _check_geometry(g, o):
    gi, og = g["info"], o["geom"]
    assert (gi["p"], gi["q"], gi["n_pad"], gi["n_grid"], gi["n_t0"]) == \
        (og.p, og.q, og.n_pad, og.n_grid, og.n_t0)


CASES = {
    # 2-min TESS-like, t0 step = cadence (q = 1), several linear tiles, ragged tail
    "tess_small": dict(n_points=4001, cadence_s=120.0, durations_h=synth.log_grid(0.5, 6, 10),
                       periods=synth.log_grid(0.5, 3.5, 300),
                       planets=[dict(P=1.3, t0=0.4, D=2.0 * HOUR, depth=3e-3, b=0.3)]),
    # 30-min Kepler-like with t0 step c/3 (q = 3) and data gaps
    "q3_gaps": dict(n_points=2500, cadence_s=1800.0, durations_h=synth.log_grid(1, 16, 16),
                    t0_step_s=600.0, gaps=((10.0, 13.0), (30.0, 31.5)),
                    periods=synth.log_grid(1.0, 20.0, 400),
                    planets=[dict(P=4.2, t0=1.0, D=4.0 * HOUR, depth=4e-3, b=0.2)]),
    # default t0 step: 1 % of the shortest duration -> s/c = 3/20 (p = 3, q = 20)
    "p3q20": dict(n_points=1500, cadence_s=120.0, durations_h=synth.log_grid(0.5, 3, 6),
                  t0_step_s=18.0, periods=synth.log_grid(0.4, 1.0, 120),
                  planets=[dict(P=0.61, t0=0.2, D=1.0 * HOUR, depth=5e-3, b=0.1)]),
    # irregular sampling: jitter, repeated cells, dropped points, per-point sigma
    "irregular": dict(n_points=3000, cadence_s=120.0, durations_h=(0.7, 1.9, 4.4), jitter=0.45,
                      drop_frac=0.1, sigma_spread=0.5, periods=synth.log_grid(0.3, 2.0, 200),
                      planets=[dict(P=0.9, t0=0.3, D=1.5 * HOUR, depth=4e-3, b=0.4)]),
    # windows longer than one shared-memory table chunk (> 2304 points)
    "long_window": dict(n_points=9000, cadence_s=60.0, durations_h=(2.0, 40.0, 61.0),
                        periods=synth.log_grid(2.6, 5.5, 60),
                        planets=[dict(P=2.9, t0=1.0, D=40.0 * HOUR, depth=2e-3, b=0.3)]),
    # times offset by 2.45e6 d (multi-year-style absolute times)
    "offset_time": dict(n_points=3000, cadence_s=120.0, durations_h=(1.0, 2.5), time_offset=2.45e6,
                        periods=synth.log_grid(0.3, 2.0, 150),
                        planets=[dict(P=0.77, t0=0.1, D=1.5 * HOUR, depth=3e-3, b=0.3)]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_small_case_parity(name):
    kw = dict(CASES[name])
    periods = kw.pop("periods")
    w = custom(seed=11, **kw)
    g, o = _run_both(w, periods)
    _check_geometry(g, o)
    ls = compare_linear(g, o, w.durations)
    ps = compare_periodic(g, o, periods)
    print(name, ls, ps)
    assert g["logl0"] == pytest.approx(o["logl0"], rel=1e-6)


def test_tiny_and_degenerate():
    """A few dozen points: one partial tile, durations longer than the data,
    a period shorter than the t0 step (null), a period longer than the grid
    (single epoch), a duration equal to a period (skipped)."""
    rng = np.random.default_rng(3)
    t = regular(40)
    e = sigmas(rng, t.size)
    f = (1 - 2e-3 * ((t > 10 * C_EXACT) & (t < 14 * C_EXACT)) + rng.normal(size=t.size) * e)
    f = f.astype(np.float32)
    durs = np.array([2.0, 5.0, 60.0]) * C_EXACT
    periods = np.array([0.5, 5.0, 7.3, 60.0, 1e4]) * C_EXACT
    args = (t, f, e, durs, synth.default_template())
    g = gpu_search(*args, periods, cadence=C_EXACT, t0_step=C_EXACT)
    o = oracle_search(*args, periods, cadence=C_EXACT, t0_step=C_EXACT)
    compare_linear(g, o, durs)
    compare_periodic(g, o, periods)
    assert np.isnan(g["periodic"]["dlogl"][0])  # P < s is null


def test_flat_data_exact_zero_and_tie_rule():
    rng = np.random.default_rng(4)
    t = regular(3000)
    e = sigmas(rng, t.size)
    f = np.ones(t.size, np.float32)
    durs = np.array([3.0, 9.5, 21.0]) * C_EXACT
    periods = synth.log_grid(30 * C_EXACT, 900 * C_EXACT, 50)
    args = (t, f, e, durs, synth.default_template())
    g = gpu_search(*args, periods, cadence=C_EXACT, t0_step=C_EXACT / 2)
    o = oracle_search(*args, periods, cadence=C_EXACT, t0_step=C_EXACT / 2)
    ok = ~np.isnan(o["dlogl"])
    assert np.all(g["dlogl"][ok] == 0.0) and np.all(g["depth"][ok] == 0.0)
    np.testing.assert_array_equal(g["periodic"]["i"], o["periodic"]["i"])
    np.testing.assert_array_equal(g["periodic"]["j"], o["periodic"]["j"])
    assert np.all(g["periodic"]["dlogl"] == 0.0)


def test_box_injection_exact_values():
    """Noiseless box transit: the cell at the injected (t0, D) gives depth =
    alpha and LR = alpha^2 sum(W) / 2 to FP32 accuracy (Sec. 2.2)."""
    rng = np.random.default_rng(2)
    t = regular(5000)
    e = sigmas(rng, t.size)
    alpha = 2.0 ** -10
    y = np.zeros(t.size, np.float32)
    y[2495:2506] = alpha
    g = gpu_search(t, y, e, [10.5 * C_EXACT], box_template(), [3000 * C_EXACT],
                   cadence=C_EXACT, t0_step=C_EXACT, flux_is_offset=True)
    i = g["info"]["n_pad"] + 2500
    w = 1.0 / e.astype(np.float64) ** 2
    B = w[2495:2506].sum()
    assert g["depth"][0, i] == pytest.approx(alpha, rel=2e-6)
    assert g["dlogl"][0, i] == pytest.approx(alpha * alpha * B / 2, rel=5e-6)
    assert int(np.nanargmax(g["dlogl"][0])) == i
    assert g["periodic"]["i"][0] == i and g["periodic"]["j"][0] == 0


def test_mask_and_flux_offset():
    w = custom(seed=5, n_points=4000, cadence_s=120.0, durations_h=(0.5, 1.5, 3.0),
               planets=[dict(P=1.1, t0=0.5, D=1.5 * HOUR, depth=3e-3, b=0.3)])
    periods = synth.log_grid(0.4, 2.5, 120)
    rng = np.random.default_rng(0)
    mask = (rng.uniform(size=(periods.size, 3)) < 0.6).astype(np.uint8)
    mask[:5] = 0  # periods with every duration masked are null
    y = (1.0 - w.flux.astype(np.float64)).astype(np.float32)
    args = (w.time, y, w.flux_err, w.durations, w.template)
    g = gpu_search(*args, periods, mask, cadence=w.cadence, t0_step=w.t0_step, flux_is_offset=True)
    o = oracle_search(*args, periods, mask, cadence=w.cadence, t0_step=w.t0_step,
                      flux_is_offset=True)
    compare_linear(g, o, w.durations)
    compare_periodic(g, o, periods)
    assert np.all(np.isnan(g["periodic"]["dlogl"][:5]))


def test_periods_with_more_epochs_than_the_offset_table():
    """Periods of 8-15 t0 steps on a 40,000-point curve have 2,700-5,000 epochs: more
    than the fold's shared offset table holds for even one period, so each is folded
    from global memory with its offsets computed in FP64 on the fly. Longer periods in
    the same launch take the table path; every period is compared with the oracle."""
    short = synth.log_grid(16.0 / 1440.0, 30.0 / 1440.0, 40)  # 8-15 steps of 2 min
    long = synth.log_grid(0.05, 2.0, 40)
    periods = np.concatenate([short, long])
    P_in = short[20]  # on the grid: an off-grid period dephases over thousands of epochs
    w = custom(seed=23, n_points=40000, cadence_s=120.0, durations_h=(0.1, 0.2, 0.3),
               planets=[dict(P=P_in, t0=0.004, D=0.2 * HOUR, depth=1e-4, b=0.2)])
    g, o = _run_both(w, periods)
    _check_geometry(g, o)
    I, s = g["info"]["n_t0"], w.t0_step
    epochs = np.floor((I + 0.5) / (short / s)) + 1
    assert epochs.min() > 2048  # beyond the table for a single period
    ls = compare_linear(g, o, w.durations)
    ps = compare_periodic(g, o, periods)
    print("fold_direct", ls, ps)
    kb = ps["best_k"][0]
    assert abs(periods[kb] - P_in) / P_in < 0.01


def test_duration_packed_short_periods_in_a_large_launch():
    """12,000 short trial periods (0.35-3.0 d at a 10-min t0 step: 51-432 phases) over five
    durations: the launch has more 8-period groups than four per block slot of the GPU, so
    each work item holds every duration, and the fold packs the phases of several durations
    into one tile (the duration-packed path) wherever that fills at least half of the lanes;
    the shortest periods take the epoch-sliced path. Durations longer than a period and a
    (duration, period) mask leave some durations out of some groups. Every period is compared
    with the oracle."""
    periods = synth.log_grid(0.35, 3.0, 12000)
    w = custom(seed=31, n_points=1296, cadence_s=1800.0, t0_step_s=600.0,
               durations_h=(1.0, 2.0, 4.0, 8.0, 12.0),
               planets=[dict(P=1.7, t0=0.6, D=3.0 * HOUR, depth=3e-3, b=0.3)])
    rng = np.random.default_rng(4)
    mask = (rng.uniform(size=(periods.size, 5)) < 0.7).astype(np.uint8)
    g, o = _run_both(w, periods, mask)
    _check_geometry(g, o)
    nph = np.ceil(periods / w.t0_step)
    assert nph.max() <= 448 and periods.size // 8 >= 4 * 2 * 152
    compare_linear(g, o, w.durations)
    ps = compare_periodic(g, o, periods)
    kb = ps["best_k"][0]
    assert abs(periods[kb] - 1.7) / 1.7 < 0.01


def test_host_buffer_api_matches_device_api():
    from paper_2503_20875_gb300 import Context, cetra_linear_search, cetra_periodic_search
    w = custom(seed=6, n_points=5000, cadence_s=120.0, durations_h=(0.5, 1.0, 2.0, 4.0),
               planets=[dict(P=1.7, t0=0.5, D=2.0 * HOUR, depth=3e-3, b=0.3)])
    periods = synth.log_grid(0.5, 3.0, 200)
    g = gpu_search(w.time, w.flux, w.flux_err, w.durations, w.template, periods,
                   cadence=w.cadence, t0_step=w.t0_step)
    ctx = Context(0)
    grid, dep, var, lr = cetra_linear_search(ctx, w.time, w.flux, w.flux_err, w.durations,
                                             w.template, cadence=w.cadence, t0_step=w.t0_step)
    np.testing.assert_array_equal(np.isnan(lr), np.isnan(g["dlogl"]))
    np.testing.assert_allclose(lr, g["dlogl"], rtol=1e-5, atol=1e-5)
    per = cetra_periodic_search(ctx, grid, periods)
    np.testing.assert_allclose(per["dlogl"], g["periodic"]["dlogl"], rtol=1e-6)
    np.testing.assert_array_equal(per["t0"], g["periodic"]["t0"])
    assert per["best_k"] == int(np.nanargmax(g["periodic"]["dlogl"]))
    grid.close()


def test_invalid_arguments_fail_cleanly_on_device():
    import torch
    from paper_2503_20875_gb300 import Context, Plan, CetraError, cetra_linear_search
    ctx = Context(0)
    t = regular(100)
    f = np.ones(t.size, np.float32)
    e = np.full(t.size, 1e-3, np.float32)
    with pytest.raises(CetraError):
        Plan(ctx, t, f, e, [-1.0], box_template())
    with pytest.raises(CetraError):
        Plan(ctx, t, f, e, [0.1], np.zeros(4, np.float32))  # zero template
    with pytest.raises(CetraError):
        cetra_linear_search(ctx, t, f, np.zeros_like(e), [0.1], box_template())
    plan = Plan(ctx, t, f, e, [4 * C_EXACT], box_template(), cadence=C_EXACT)
    from paper_2503_20875_gb300 import cetra_linear_device
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(CetraError):
        cetra_linear_device(ctx, plan, small)  # workspace too small
    torch.cuda.synchronize()  # the context is still healthy
    g = gpu_search(t, f, e, [4 * C_EXACT], box_template(), [50 * C_EXACT], cadence=C_EXACT)
    assert np.all(np.nan_to_num(g["dlogl"]) == 0.0)


# ----------------------------------------------------------------------------- full sizes


def test_full_tess_2min_27d():
    """27 d at 2-min cadence, 10 durations, 2,000 periods: every cell, every period."""
    w = synth.make_workload("tess_2min_27d")
    g, o = _run_both(w)
    _check_geometry(g, o)
    ls = compare_linear(g, o, w.durations)
    ps = compare_periodic(g, o, w.periods)
    print("tess_2min_27d", ls, ps)
    k = ps["best_k"][0]
    assert abs(w.periods[k] - 3.7) / 3.7 < 0.01  # the injected planet is recovered


def test_full_tess_20s_27d_sampled_periods():
    """27 d at 20-s cadence: the whole linear grid; the fold on every 50th
    period plus the 200 periods around the best one."""
    w = synth.make_workload("tess_20s_27d")
    g_all = gpu_search(w.time, w.flux, w.flux_err, w.durations, w.template, w.periods,
                       cadence=w.cadence, t0_step=w.t0_step)
    kbest = int(np.nanargmax(g_all["periodic"]["dlogl"]))
    sel = np.unique(np.concatenate([np.arange(0, w.periods.size, 50),
                                    np.arange(max(0, kbest - 100), min(w.periods.size, kbest + 100))]))
    o = oracle_search(w.time, w.flux, w.flux_err, w.durations, w.template, w.periods[sel],
                      cadence=w.cadence, t0_step=w.t0_step)
    _check_geometry(g_all, o)
    ls = compare_linear(g_all, o, w.durations)
    g_sel = dict(g_all)
    g_sel["periodic"] = {k: v[sel] for k, v in g_all["periodic"].items()}
    ps = compare_periodic(g_sel, o, w.periods[sel])
    print("tess_20s_27d", ls, ps)
    assert abs(w.periods[kbest] - 11.3) / 11.3 < 0.01 or abs(w.periods[kbest] - 5.1) / 5.1 < 0.01


def test_full_kepler_1min_4yr_sampled_periods():
    """4-yr baseline at 1-min cadence (2.1 M points, absolute times + 2.45e6 d),
    30 durations: the whole linear grid; the fold on every 1000th period plus the
    41 periods around the injected 365-d transit. Multi-year tolerance 1e-4."""
    w = synth.make_workload("kepler_1min_4yr")
    k365 = int(np.argmin(np.abs(w.periods - 365.0)))
    sel = np.unique(np.concatenate([np.arange(0, w.periods.size, 1000),
                                    np.arange(k365 - 20, k365 + 21)]))
    P = w.periods[sel]
    g = gpu_search(w.time, w.flux, w.flux_err, w.durations, w.template, P, cadence=w.cadence,
                   t0_step=w.t0_step)
    o = oracle_search(w.time, w.flux, w.flux_err, w.durations, w.template, P,
                      cadence=w.cadence, t0_step=w.t0_step)
    _check_geometry(g, o)
    ls = compare_linear(g, o, w.durations, r_flat=1e-4)
    ps = compare_periodic(g, o, P, r_flat=1e-4, r_low=1e-4)
    print("kepler_1min_4yr", ls, ps)


# ----------------------------------------------------------------------------- precision form


@pytest.mark.parametrize("name", ["tess_small", "q3_gaps", "p3q20", "long_window"])
def test_kahan_small_case_parity(name):
    """CETRA_FP32_KAHAN: compensated window and fold sums, same bounds as plain."""
    kw = dict(CASES[name])
    periods = kw.pop("periods")
    w = custom(seed=11, **kw)
    args = (w.time, w.flux, w.flux_err, w.durations, w.template, periods)
    g = gpu_search(*args, cadence=w.cadence, t0_step=w.t0_step, precision="kahan")
    o = oracle_search(*args, cadence=w.cadence, t0_step=w.t0_step)
    _check_geometry(g, o)
    print(name, "kahan", compare_linear(g, o, w.durations), compare_periodic(g, o, periods))


def _max_rel(a, b, sel):
    return float(np.max(np.abs(a[sel].astype(np.float64) - b[sel]) / np.abs(b[sel]), initial=0.0))


def test_kahan_vs_plain_error_on_4yr_baseline():
    """The precision form on the 4-yr workload: both forms meet the bound, and the
    compensated sums are at least as close to the FP64 oracle as the plain ones."""
    w = synth.make_workload("kepler_1min_4yr")
    k365 = int(np.argmin(np.abs(w.periods - 365.0)))
    P = w.periods[np.unique(np.concatenate([np.arange(0, w.periods.size, 2000),
                                            np.arange(k365 - 5, k365 + 6)]))]
    args = (w.time, w.flux, w.flux_err, w.durations, w.template, P)
    kw = dict(cadence=w.cadence, t0_step=w.t0_step)
    o = oracle_search(*args, **kw)
    plain = gpu_search(*args, **kw)
    kahan = gpu_search(*args, **kw, precision="kahan")
    sig = ~np.isnan(o["dlogl"]) & (o["dlogl"] >= 25)
    ok = ~np.isnan(o["dlogl"])
    report = {}
    for name, g in (("plain", plain), ("kahan", kahan)):
        compare_linear(g, o, w.durations, r_flat=1e-4)
        compare_periodic(g, o, P, r_flat=1e-4, r_low=1e-4)
        report[name] = {"lin_sig": _max_rel(g["dlogl"], o["dlogl"], sig),
                        "depth_all": _max_rel(g["depth"], o["depth"], ok & (np.abs(o["depth"]) > 0)),
                        "per": _max_rel(g["periodic"]["dlogl"], o["periodic"]["dlogl"],
                                        ~np.isnan(o["periodic"]["dlogl"]))}
    print("precision form (max relative error vs the FP64 oracle)", report)
    assert report["kahan"]["lin_sig"] <= report["plain"]["lin_sig"] + 2e-7
    assert report["kahan"]["per"] <= report["plain"]["per"] + 2e-7
