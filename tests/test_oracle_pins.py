"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests re-calls an oracle routine to produce its expected value.
Each one checks the oracle against a closed form, a brute-force maximisation
of the full likelihood (Eq. 1) over the raw observations, an invariant, a
special case, or a fact the paper prints (fixtures under tests/golden/).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests._cases import C_EXACT, regular, sigmas, box_template

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run(time, flux, err, durations, tmpl, periods=None, **kw):
    return oracle.search(time, flux, err, durations, tmpl, periods, **kw)


# --------------------------------------------------------------------------- geometry


def test_default_cadence_is_median_of_diffs():
    rng = np.random.default_rng(3)
    t = np.sort(rng.uniform(0, 5, 301))
    f = np.ones_like(t, dtype=np.float32)
    e = np.full(t.size, 1e-3, np.float32)
    g = oracle.geometry(t, f, e, [0.1])
    d = np.diff(t - t.min())
    assert g.cadence == pytest.approx(float(np.median(d[d > 0])), rel=0, abs=0)


def test_padding_and_grid_extent():
    t = regular(1000)
    f = np.ones(t.size, np.float32)
    e = np.full(t.size, 1e-3, np.float32)
    for dmax_c in (3.5, 10.0, 10.25, 64.0):
        g = oracle.geometry(t, f, e, [1.5 * C_EXACT, dmax_c * C_EXACT], cadence=C_EXACT,
                            t0_step=C_EXACT)
        # Sec. 2.1.1: padded by half the longest duration at both ends
        assert g.n_pad == math.ceil(dmax_c / 2)
        assert g.n_grid == 2 * g.n_pad + 1000
        # R5: t0 grid spans the padded grid at step s = c
        assert g.n_t0 == g.n_grid


@pytest.mark.parametrize("ratio,pq", [(1.0, (1, 1)), (0.15, (3, 20)), (1 / 3, (1, 3)),
                                      (2.0, (2, 1)), (0.5, (1, 2))])
def test_t0_step_realised_as_rational(ratio, pq):
    t = regular(200)
    f = np.ones(t.size, np.float32)
    e = np.full(t.size, 1e-3, np.float32)
    g = oracle.geometry(t, f, e, [4 * C_EXACT], cadence=C_EXACT, t0_step=ratio * C_EXACT)
    assert (g.p, g.q) == pq
    assert g.t0_step == pytest.approx(ratio * C_EXACT, rel=1e-12)


def test_t0_step_default_is_one_percent_of_min_duration():
    t = regular(200)
    f = np.ones(t.size, np.float32)
    e = np.full(t.size, 1e-3, np.float32)
    g = oracle.geometry(t, f, e, [20 * C_EXACT, 40 * C_EXACT], cadence=C_EXACT)
    assert g.t0_step == pytest.approx(0.2 * C_EXACT, rel=1e-12)  # 1 % of 20 c
    assert (g.p, g.q) == (1, 5)


def test_irrational_step_best_approximation():
    t = regular(200)
    f = np.ones(t.size, np.float32)
    e = np.full(t.size, 1e-3, np.float32)
    r = math.pi / 10
    g = oracle.geometry(t, f, e, [4 * C_EXACT], cadence=C_EXACT, t0_step=r * C_EXACT)
    best = min(((abs(round(q * r) / q - r), q) for q in range(1, 65)))
    assert g.q == best[1] and g.p == round(best[1] * r)


# --------------------------------------------------------------------------- resampling


def test_resample_inverse_variance_combination():
    # two observations in one cell, one in another, the rest null
    t = np.array([0.0, 10 * C_EXACT + 0.1 * C_EXACT, 10 * C_EXACT - 0.2 * C_EXACT, 20 * C_EXACT])
    f = np.array([1.0, 1.0 - 2e-3, 1.0 - 4e-3, 1.0], np.float32)
    e = np.array([1e-3, 1e-3, 2e-3, 1e-3], np.float32)
    g = oracle.geometry(t, f, e, [2 * C_EXACT], cadence=C_EXACT, t0_step=C_EXACT)
    y, w = oracle.resample(t, f, e, g)
    k = g.n_pad + 10
    w1, w2 = 1 / float(e[1]) ** 2, 1 / float(e[2]) ** 2
    y1, y2 = 1 - float(f[1]), 1 - float(f[2])
    assert w[k] == pytest.approx(w1 + w2, rel=1e-15)
    assert y[k] == pytest.approx((w1 * y1 + w2 * y2) / (w1 + w2), rel=1e-14)
    assert np.count_nonzero(w) == 3
    assert w[g.n_pad] > 0 and w[g.n_pad + 20] > 0


def test_logl0_matches_eq1_at_zero_depth():
    rng = np.random.default_rng(5)
    t = regular(300)
    e = sigmas(rng, t.size)
    f = (1 + rng.normal(size=t.size) * e).astype(np.float32)
    r = run(t, f, e, [4 * C_EXACT], box_template(), cadence=C_EXACT, t0_step=C_EXACT)
    y = 1.0 - f.astype(np.float64)
    s2 = e.astype(np.float64) ** 2
    expect = np.sum(-0.5 * y * y / s2 - 0.5 * np.log(2 * np.pi * s2))
    assert r["logl0"] == pytest.approx(expect, rel=1e-12)


# --------------------------------------------------------------------------- template


def test_template_identity_resampling_and_normalisation():
    tm = (np.arange(1025) * 3).astype(np.float32)
    T = oracle.template(tm, 1025)
    np.testing.assert_array_equal(T, tm.astype(np.float64) / tm.max())


def test_template_linear_interpolation_midpoints():
    # a 3-sample model resampled to 5 samples: interpolation at the midpoints
    T = oracle.template(np.array([0.0, 1.0, 0.5], np.float32), 5)
    np.testing.assert_allclose(T, [0.0, 0.5, 1.0, 0.75, 0.5], rtol=0, atol=1e-15)


def test_template_nn_error_matches_figure_1():
    fx = json.load(open(os.path.join(GOLDEN, "template_nn_error.json")))
    dense = synth.ld_transit_template(16385, b=0.32, p=0.03, u1=0.4804, u2=0.1867)
    T = oracle.template(dense.astype(np.float32), fx["L"])
    x_dense = np.arange(dense.size) / (dense.size - 1)
    x_l = np.arange(fx["L"]) / (fx["L"] - 1)
    nearest = np.abs(x_dense[:, None] - x_l[None, :]).argmin(axis=1)
    err = np.abs(dense - T[nearest])
    assert fx["max_error_approx"] / 3 <= err.max() <= fx["max_error_approx"] * 3
    assert fx["mean_error_approx"] / 3 <= err.mean() <= fx["mean_error_approx"] * 3


# --------------------------------------------------------------------------- linear search


def _curve(seed, n=600, gaps=((150, 190),), dup=True):
    rng = np.random.default_rng(seed)
    k = np.arange(n)
    keep = np.ones(n, bool)
    for lo, hi in gaps:
        keep[lo:hi] = False
    k = k[keep]
    t = k * C_EXACT + rng.uniform(-0.3, 0.3, k.size) * C_EXACT
    if dup:  # a second observation in some cells
        extra = rng.choice(k, size=k.size // 5, replace=False)
        t = np.concatenate([t, extra * C_EXACT + rng.uniform(-0.3, 0.3, extra.size) * C_EXACT])
    e = sigmas(rng, t.size)
    f = (1 + rng.normal(size=t.size) * e).astype(np.float32)
    return t, f, e


def test_linear_two_pass_equals_closed_form():
    """Eq. 2 evaluated at the pass-1 depth equals Delta^2 / (2 var) (P1)."""
    t, f, e = _curve(1)
    durs = np.array([3.3, 7.9, 12.25, 30.0]) * C_EXACT
    r = run(t, f, e, durs, synth.default_template(), cadence=C_EXACT, t0_step=C_EXACT / 3)
    lr, dep, var = r["dlogl"], r["depth"], r["depth_var"]
    ok = ~np.isnan(lr)
    scale = np.sum(r["w_grid"] * r["y_grid"] ** 2)
    np.testing.assert_allclose(lr[ok], 0.5 * dep[ok] ** 2 / var[ok], rtol=0, atol=1e-12 * scale)
    assert np.all(lr[ok] >= -1e-12 * scale)
    # nulls exactly where the window holds no data (the gap is longer than 30 c)
    assert np.isnan(lr).any() and ok.any()


def test_box_template_noiseless_injection():
    """y = alpha on the window of (t_i, D_j): Delta = alpha, LR = alpha^2 / (2 var) (P2)."""
    rng = np.random.default_rng(2)
    t = regular(400)
    e = sigmas(rng, t.size)
    alpha = 2.0 ** -10
    y = np.zeros(t.size, np.float32)
    y[195:206] = alpha  # D = 10.5 c centred on point 200 covers points 195..205
    r = run(t, y, e, [10.5 * C_EXACT], box_template(), cadence=C_EXACT, t0_step=C_EXACT,
            flux_is_offset=True)
    g = r["geom"]
    assert g.n_pad == 6
    i = g.n_pad + 200
    w = 1.0 / e.astype(np.float64) ** 2
    var = 1.0 / w[195:206].sum()
    assert r["depth"][0, i] == pytest.approx(alpha, rel=1e-14)
    assert r["depth_var"][0, i] == pytest.approx(var, rel=1e-14)
    assert r["dlogl"][0, i] == pytest.approx(alpha * alpha / (2 * var), rel=1e-12)
    assert np.nanargmax(r["dlogl"][0]) == i


@pytest.mark.parametrize("reverse", [False, True])
def test_shaped_template_exact_samples(reverse):
    """A ramp template whose samples land exactly on grid points: the data built
    from those samples is recovered with Delta = alpha exactly, and the edge
    points (x = 0 and x = 1) are inside the window (R4)."""
    rng = np.random.default_rng(4)
    L = 1025
    tm = (0.25 + 0.75 * np.arange(L) / (L - 1)).astype(np.float32)
    if reverse:
        tm = tm[::-1].copy()
    t = regular(300)
    e = sigmas(rng, t.size)
    alpha = 2.0 ** -9
    y = np.zeros(t.size, np.float32)
    for u in range(9):  # D = 8 c: points 146..154, x = u / 8, sample index 128 u
        y[146 + u] = alpha * tm[128 * u]
    r = run(t, y, e, [8 * C_EXACT], tm, L=L, cadence=C_EXACT, t0_step=C_EXACT,
            flux_is_offset=True)
    i = r["geom"].n_pad + 150
    w = 1.0 / e.astype(np.float64) ** 2
    m = tm[128 * np.arange(9)].astype(np.float64)
    B = np.sum(m * m * w[146:155])
    assert r["depth"][0, i] == pytest.approx(alpha, rel=1e-14)
    assert r["depth_var"][0, i] == pytest.approx(1.0 / B, rel=1e-14)
    assert r["dlogl"][0, i] == pytest.approx(alpha * alpha * B / 2, rel=1e-12)


def test_flat_data_gives_zero():
    """y = 0 everywhere: Delta = 0 and LR = 0 exactly, linear and periodic (P3)."""
    rng = np.random.default_rng(6)
    t = regular(500)
    e = sigmas(rng, t.size)
    f = np.ones(t.size, np.float32)
    P = np.array([37, 50.5, 91]) * C_EXACT
    r = run(t, f, e, [3 * C_EXACT, 9.5 * C_EXACT], synth.default_template(), P,
            cadence=C_EXACT, t0_step=C_EXACT / 2)
    ok = ~np.isnan(r["dlogl"])
    assert np.all(r["dlogl"][ok] == 0.0) and np.all(r["depth"][ok] == 0.0)
    per = r["periodic"]
    assert np.all(per["dlogl"] == 0.0) and np.all(per["depth"] == 0.0)
    # ties everywhere: the smallest duration index, then the smallest valid phase
    assert np.all(per["j"] == 0)


def _brute_lr(y, s2, model):
    """max_Z sum[-1/2 (Z m - y)^2 / s2] - sum[-1/2 y^2 / s2] by golden-section search."""
    def logl(z):
        return -0.5 * np.sum((z * model - y) ** 2 / s2)
    if not np.any(model != 0):
        return np.nan
    lo, hi = -1.0, 1.0
    gr = (math.sqrt(5) - 1) / 2
    a, b = lo + (1 - gr) * (hi - lo), lo + gr * (hi - lo)
    fa, fb = logl(a), logl(b)
    for _ in range(200):
        if fa < fb:
            lo, a, fa = a, b, fb
            b = lo + gr * (hi - lo)
            fb = logl(b)
        else:
            hi, b, fb = b, a, fa
            a = lo + (1 - gr) * (hi - lo)
            fa = logl(a)
    z = 0.5 * (lo + hi)
    return logl(z) - logl(0.0)


def _tiny_curve(seed, n_cells=56, holes=(20, 21, 22, 40)):
    rng = np.random.default_rng(seed)
    cells = np.array([k for k in range(n_cells) if k not in holes])
    t = cells * C_EXACT + rng.uniform(-0.3, 0.3, cells.size) * C_EXACT
    t = np.concatenate([t, cells[::7] * C_EXACT + 0.2 * C_EXACT])  # doubled cells
    e = sigmas(rng, t.size, 0.5e-3, 3e-3)
    f = (1 - 1.5e-3 * ((t > 30 * C_EXACT) & (t < 36 * C_EXACT))
         + rng.normal(size=t.size) * e).astype(np.float32)
    return t, f, e


def test_linear_brute_force_full_likelihood():
    """LR_ij equals the maximised full-curve Eq. 1 minus Eq. 1 at zero depth,
    over the raw observations, box model (P5): checks the window truncation,
    the MLE and the resampling combination rule."""
    t, f, e = _tiny_curve(7)
    durs = np.array([3.5, 6.5]) * C_EXACT
    r = run(t, f, e, durs, box_template(), cadence=C_EXACT, t0_step=C_EXACT)
    g = r["geom"]
    y = 1.0 - f.astype(np.float64)
    s2 = e.astype(np.float64) ** 2
    cell_time = np.floor((t - t.min()) / C_EXACT + 0.5) * C_EXACT  # nearest grid time
    for j, D in enumerate(durs):
        for i in range(g.n_t0):
            ti = (i - g.n_pad) * C_EXACT
            model = (np.abs(cell_time - ti) <= D / 2).astype(np.float64)
            bf = _brute_lr(y, s2, model)
            got = r["dlogl"][j, i]
            if np.isnan(bf):
                assert np.isnan(got)
            else:
                assert got == pytest.approx(bf, rel=1e-8, abs=1e-9)


def test_periodic_brute_force_full_likelihood():
    """LR_k and its argmax equal the brute-force maximum over (t_i, D_j) of the
    common-depth periodic model fitted to all raw observations (P5)."""
    t, f, e = _tiny_curve(8, n_cells=120, holes=(50, 51, 52, 53, 90))
    durs = np.array([2.5, 5.5]) * C_EXACT
    periods = np.array([17.0, 23.0, 40.0]) * C_EXACT  # exact multiples of s = c
    r = run(t, f, e, durs, box_template(), periods, cadence=C_EXACT, t0_step=C_EXACT)
    g = r["geom"]
    y = 1.0 - f.astype(np.float64)
    s2 = e.astype(np.float64) ** 2
    cell_time = np.floor((t - t.min()) / C_EXACT + 0.5) * C_EXACT
    per = r["periodic"]
    for k, P in enumerate(periods):
        m = int(round(P / C_EXACT))
        best, arg = -np.inf, None
        for j, D in enumerate(durs):
            for i in range(min(m, g.n_t0)):
                model = np.zeros(t.size)
                e_ = 0
                while i + e_ * m < g.n_t0:
                    tc = (i + e_ * m - g.n_pad) * C_EXACT
                    model[np.abs(cell_time - tc) <= D / 2] = 1.0
                    e_ += 1
                v = _brute_lr(y, s2, model)
                if not np.isnan(v) and v > best + 1e-9 * abs(v):
                    best, arg = v, (i, j)
        assert per["dlogl"][k] == pytest.approx(best, rel=1e-8)
        assert (per["i"][k], per["j"][k]) == arg


def test_phases_extend_to_ceil_of_period():
    """R6: for P = 20.5 s the phases are i = 0..20; a transit seen only from
    phase 20 (its cell has no earlier epoch) must be found there."""
    rng = np.random.default_rng(15)
    t = regular(200)
    e = sigmas(rng, t.size)
    y = (rng.normal(size=t.size) * e).astype(np.float32)
    # D = 3 c -> n_pad = 2; cell 20 is data point 18; its window covers points 17..19
    y[17:20] += 0.05
    r = run(t, y, e, [3 * C_EXACT], box_template(), [20.5 * C_EXACT], cadence=C_EXACT,
            t0_step=C_EXACT, flux_is_offset=True)
    assert r["geom"].n_pad == 2
    assert r["periodic"]["i"][0] == 20


def test_period_shorter_than_t0_step_is_null():
    """R12: P < s folds a window onto itself; such periods are null."""
    t, f, e = _curve(16, n=200)
    r = run(t, f, e, [0.3 * C_EXACT], box_template(), [0.5 * C_EXACT, 3.0 * C_EXACT],
            cadence=C_EXACT, t0_step=C_EXACT)
    per = r["periodic"]
    assert np.isnan(per["dlogl"][0]) and per["i"][0] == -1 and per["j"][0] == -1
    assert not np.isnan(per["dlogl"][1])


def test_single_epoch_fold_equals_linear():
    """P longer than the t0 grid: every phase has one epoch, so the per-period
    maximum is the linear-search maximum over i < ceil(P/s) (P4)."""
    t, f, e = _curve(9, n=400)
    durs = np.array([3.0, 6.0, 11.0]) * C_EXACT
    r = run(t, f, e, durs, synth.default_template(), [1e3, 2e3], cadence=C_EXACT,
            t0_step=C_EXACT / 4)
    lr = r["dlogl"]
    flat = np.where(np.isnan(lr), -np.inf, lr)
    j, i = np.unravel_index(np.argmax(flat), flat.shape)
    per = r["periodic"]
    for k in range(2):
        assert per["dlogl"][k] == pytest.approx(lr[j, i], rel=1e-12)
        assert (per["j"][k], per["i"][k]) == (j, i)
        assert per["depth"][k] == pytest.approx(r["depth"][j, i], rel=1e-12)
        assert per["depth_var"][k] == pytest.approx(r["depth_var"][j, i], rel=1e-12)


def test_periodic_closed_form_and_cauchy_schwarz():
    """Eq. 4 summed at the common depth equals Z^2 / (2 var_Z) (P1), and the
    periodic LR never exceeds the sum of its epochs' LR (Cauchy-Schwarz)."""
    t, f, e = _curve(10, n=900, gaps=((300, 340),))
    durs = np.array([4.0, 9.0]) * C_EXACT
    periods = synth.log_grid(20 * C_EXACT, 300 * C_EXACT, 60)
    r = run(t, f, e, durs, synth.default_template(), periods, cadence=C_EXACT, t0_step=C_EXACT)
    per = r["periodic"]
    np.testing.assert_allclose(per["dlogl"], 0.5 * per["depth"] ** 2 / per["depth_var"],
                               rtol=1e-9)
    lr = np.nan_to_num(r["dlogl"], nan=0.0)
    g = r["geom"]
    for k, P in enumerate(periods):
        j, i = per["j"][k], per["i"][k]
        Ps = P / g.t0_step
        cells = [i + int(math.floor(e_ * Ps + 0.5)) for e_ in range(int(g.n_t0 / Ps) + 2)]
        cells = [c for c in cells if c < g.n_t0]
        assert per["dlogl"][k] <= lr[j, cells].sum() * (1 + 1e-12)


def test_duration_not_shorter_than_period_is_skipped_and_mask():
    t, f, e = _curve(11, n=500)
    durs = np.array([3.0, 40.0]) * C_EXACT
    periods = np.array([30.0, 60.0]) * C_EXACT
    r = run(t, f, e, durs, synth.default_template(), periods, cadence=C_EXACT, t0_step=C_EXACT)
    per = r["periodic"]
    assert per["j"][0] == 0  # D = 40 c >= P = 30 c is not evaluated
    # D == P is not evaluated either (Sec. 2.3: durations must be smaller than the period)
    y = np.zeros(t.size, np.float32)
    y[(t > 100 * C_EXACT) & (t < 120 * C_EXACT)] = 1e-2
    eq = run(t, y, e, np.array([2.0, 30.0]) * C_EXACT, box_template(), [30.0 * C_EXACT],
             cadence=C_EXACT, t0_step=C_EXACT, flux_is_offset=True)
    assert eq["periodic"]["j"][0] == 0
    r1 = run(t, f, e, durs[:1], synth.default_template(), periods, cadence=C_EXACT,
             t0_step=C_EXACT)
    mask = np.array([[1, 1], [1, 0]], np.uint8)
    r2 = run(t, f, e, durs, synth.default_template(), periods, cadence=C_EXACT, t0_step=C_EXACT,
             mask=mask)
    # with the long duration masked out at P = 60 c both periods use D = 3 c only;
    # the linear arrays for j = 0 are identical, so the fold is too
    assert r2["periodic"]["dlogl"][1] == pytest.approx(r1["periodic"]["dlogl"][1], rel=1e-13)
    assert r2["periodic"]["j"][1] == 0


# --------------------------------------------------------------------------- invariants


def test_scaling_invariants():
    """y -> 2y: Delta -> 2 Delta, LR -> 4 LR; sigma -> 2 sigma: LR -> LR / 4 (P6)."""
    rng = np.random.default_rng(12)
    t = regular(500)
    e = sigmas(rng, t.size)
    y = (rng.normal(size=t.size) * e).astype(np.float32)
    durs = np.array([3.0, 7.5]) * C_EXACT
    P = synth.log_grid(20 * C_EXACT, 200 * C_EXACT, 25)
    kw = dict(cadence=C_EXACT, t0_step=C_EXACT, flux_is_offset=True)
    base = run(t, y, e, durs, synth.default_template(), P, **kw)
    sc = run(t, 2 * y, e, durs, synth.default_template(), P, **kw)
    es = run(t, y, 2 * e, durs, synth.default_template(), P, **kw)
    ok = ~np.isnan(base["dlogl"])
    np.testing.assert_allclose(sc["depth"][ok], 2 * base["depth"][ok], rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(sc["dlogl"][ok], 4 * base["dlogl"][ok], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(es["dlogl"][ok], base["dlogl"][ok] / 4, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(sc["periodic"]["dlogl"], 4 * base["periodic"]["dlogl"], rtol=1e-9)
    np.testing.assert_array_equal(sc["periodic"]["i"], base["periodic"]["i"])


def test_null_points_and_permutation_change_nothing():
    """Invalid observations are dropped; a lone null grid point is invisible;
    the order of the observations does not matter (P6, Sec. 2.2)."""
    t, f, e = _curve(13, n=400, dup=False)
    durs = np.array([3.0, 8.0]) * C_EXACT
    P = synth.log_grid(15 * C_EXACT, 150 * C_EXACT, 20)
    kw = dict(cadence=C_EXACT, t0_step=C_EXACT)
    base = run(t, f, e, durs, synth.default_template(), P, **kw)
    rng = np.random.default_rng(0)
    tb = np.concatenate([t, rng.uniform(t.min(), t.max(), 30)])
    fb = np.concatenate([f, np.full(30, np.nan, np.float32)])
    eb = np.concatenate([e, np.full(30, 1e-3, np.float32)])
    fb[-10:] = 1.0
    eb[-10:] = np.inf
    eb[-5:] = 0.0
    perm = rng.permutation(tb.size)
    alt = run(tb[perm], fb[perm], eb[perm], durs, synth.default_template(), P, **kw)
    np.testing.assert_array_equal(np.isnan(base["dlogl"]), np.isnan(alt["dlogl"]))
    np.testing.assert_array_equal(np.nan_to_num(base["dlogl"]), np.nan_to_num(alt["dlogl"]))
    for key in ("dlogl", "i", "j", "depth"):
        np.testing.assert_array_equal(base["periodic"][key], alt["periodic"][key])


def test_time_offset_keeps_indices():
    """Adding 2.45e6 d to every time leaves every index decision unchanged (P6)."""
    t, f, e = _curve(14, n=500, dup=False)
    durs = np.array([3.0, 8.0]) * C_EXACT
    P = synth.log_grid(15 * C_EXACT, 150 * C_EXACT, 20)
    kw = dict(cadence=C_EXACT, t0_step=C_EXACT)
    base = run(t, f, e, durs, synth.default_template(), P, **kw)
    off = run(t + 2.45e6, f, e, durs, synth.default_template(), P, **kw)
    np.testing.assert_allclose(np.nan_to_num(off["dlogl"]), np.nan_to_num(base["dlogl"]),
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(off["periodic"]["i"], base["periodic"]["i"])
    np.testing.assert_array_equal(off["periodic"]["j"], base["periodic"]["j"])
    np.testing.assert_allclose(off["periodic"]["t0"] - 2.45e6, base["periodic"]["t0"], atol=1e-8)


# --------------------------------------------------------------------------- the paper's example


def test_toy_example_of_figures_2_and_3():
    fx = json.load(open(os.path.join(GOLDEN, "toy_example.json")))["facts"]
    rng = np.random.default_rng(20)
    cad = 1.0 / 48
    t = np.arange(int(60 / cad)) * cad
    D = fx["transit_duration_d"]
    planets = [dict(P=np.inf, t0=tc, D=D, depth=fx["transit_depth"], b=0.32)
               for tc in fx["transit_mid_times_d"]]
    y = synth.inject_transits(t, planets)
    e = np.full(t.size, 100e-6, np.float32)
    f = (1 - y + rng.normal(size=t.size) * 100e-6).astype(np.float32)
    durs = np.array([3.0, 4.0, 5.0, 6.0, 7.0])
    periods = synth.log_grid(6.0, 45.0, 400)
    r = run(t, f, e, durs, synth.default_template(), periods, cadence=cad, t0_step=0.05)
    g = r["geom"]
    # linear search: the best single windows sit on the injected transits with D = 5 d
    lr = np.nan_to_num(r["dlogl"], nan=-np.inf)
    j, i = np.unravel_index(np.argmax(lr), lr.shape)
    t_i = g.t_ref + (i * g.p - g.n_pad * g.q) * g.cadence / g.q
    assert durs[j] == D
    assert min(abs(t_i - tc) for tc in fx["transit_mid_times_d"]) <= 0.05
    assert r["depth"][j, i] == pytest.approx(fx["transit_depth"], rel=0.05)
    # periodic search: peak at 20 d, lower peaks at the 10-d and 40-d aliases
    per = r["periodic"]["dlogl"]
    kbest = int(np.argmax(per))
    assert abs(periods[kbest] - fx["true_period_d"]) <= 0.01 * fx["true_period_d"]
    # the reported reference time is a transit mid-time of the injected train
    t0 = r["periodic"]["t0"][kbest]
    assert min(abs(t0 - tc) for tc in fx["transit_mid_times_d"]) <= 0.1
    assert r["periodic"]["duration"][kbest] == D
    for alias in fx["alias_periods_d"]:
        near = np.abs(periods - alias) <= 0.01 * alias
        assert per[near].max() < per[kbest]
        assert per[near].max() > np.median(per)


def test_cell_evaluators_agree_with_full_search():
    """The per-cell entry points (used for sampled parity at full sizes and for
    epsilon-tie checks) return exactly what the full search computes."""
    t, f, e = _curve(17, n=700)
    durs = np.array([3.0, 8.0, 13.0]) * C_EXACT
    P = synth.log_grid(20 * C_EXACT, 300 * C_EXACT, 30)
    r = run(t, f, e, durs, synth.default_template(), P, cadence=C_EXACT, t0_step=C_EXACT / 3,
            with_kappa=True)
    g = r["geom"]
    rng = np.random.default_rng(1)
    jj = rng.integers(0, 3, 500)
    ii = rng.integers(0, g.n_t0, 500)
    d, v, l, k = oracle.linear_cells(g, r["y_grid"], r["w_grid"], durs, r["T"], jj, ii)
    np.testing.assert_array_equal(d, r["depth"][jj, ii])
    np.testing.assert_array_equal(l, r["dlogl"][jj, ii])
    np.testing.assert_array_equal(k, r["kappa"][jj, ii])
    per = r["periodic"]
    lr, z, zv = oracle.periodic_at(g, r["depth"], r["depth_var"], r["dlogl"], P, per["i"], per["j"])
    np.testing.assert_array_equal(lr, per["dlogl"])
    np.testing.assert_array_equal(z, per["depth"])


def test_batch_period_grid():
    """The batched search's grid P_k = pmin ratio^k: matches the closed form within
    the rounding of square-and-multiply (each squaring doubles the relative error of
    the running power: at most about (k + 2 log2 k + 2) u), is increasing, and stops
    at the last period <= pmax."""
    u = 2.0 ** -53
    for pmin, ratio, pmax in ((0.5, 1.0 + 1 / 48 / 340, 180.0), (1.0, 1.002, 42.5), (3.0, 2.0, 3.0)):
        P = oracle.period_grid(pmin, ratio, pmax)
        k = np.arange(P.size)
        exact = pmin * ratio ** k
        bound = (k + 2 * np.log2(k + 1) + 4) * u * exact
        assert np.all(np.abs(P - exact) <= bound)
        assert np.all(np.diff(P) > 0) and P[-1] <= pmax
        assert pmin * ratio ** P.size > pmax * (1 - 1e-12)
