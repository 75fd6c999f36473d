"""Host bookkeeping of the learned period-interval proposal (no GPU): transit labels on the
t0 grid, bin widths, valid spans and the upper interval edge."""
import math

import numpy as np
import pytest

from paper_2503_20875_gb300 import proposal
from paper_2503_20875_gb300.api import batch_period_grid

INFO = dict(cadence=0.01, t0_step=0.02, p=2, q=1, n_pad=5)


def _brute_labels(t_ref, I, planets, n_bins):
    """Label every t0 cell by its own time (t_i = t_ref + i s - n_pad c), then max-pool."""
    s, c = INFO["t0_step"], INFO["cadence"]
    width = (I + n_bins - 1) // n_bins
    out = np.zeros(n_bins, np.float32)
    for i in range(I):
        t = t_ref + i * s - INFO["n_pad"] * c
        for pl in planets:
            n = round((t - pl["t0"]) / pl["P"])
            if any(abs(t - (pl["t0"] + m * pl["P"])) <= 0.5 * pl["D"] + 1e-12
                   for m in (n - 1, n, n + 1)):
                out[i // width] = 1.0
    return out


@pytest.mark.parametrize("t_ref,I,n_bins", [(0.0, 1000, 100), (12.3, 777, 64), (5.0, 50, 256)])
def test_labels_match_cell_by_cell(t_ref, I, n_bins):
    planets = [dict(P=3.0, t0=t_ref + 1.0, D=0.1), dict(P=2.2, t0=t_ref - 7.05, D=0.23)]
    geo = [(t_ref, 0.5, 1.001, 10, I, 0), (t_ref, 0.5, 1.001, 0, 0, 2)]
    got = proposal.labels(geo, INFO, [planets, planets], n_bins)
    np.testing.assert_array_equal(got[0], _brute_labels(t_ref, I, planets, n_bins))
    assert not got[1].any()  # a curve without t0 cells has no labels


def test_bin_days_and_period_max():
    geo = [(0.0, 0.5, 1.001, 100, 1000, 0), (0.0, 0.5, 1.002, 0, 0, 13), (0.0, 0.7, 1.01, 3, 9000, 13)]
    bw = proposal.bin_days(geo, INFO, 4096)
    np.testing.assert_allclose(bw, [1 * 0.02, 0.0, 3 * 0.02])
    pmax = proposal.period_max(geo)
    assert pmax >= max(batch_period_grid(0.5, 1.001, 100)[-1], batch_period_grid(0.7, 1.01, 3)[-1])
    assert pmax <= 0.7 * 1.01 ** 2 * (1 + 1e-8)


def test_n_valid_counts_occupied_bins():
    geo = [(0.0, 0.5, 1.001, 10, I, 0) for I in (1000, 777, 50, 4097, 1)] + \
          [(0.0, 0.5, 1.001, 0, 0, 0)]
    for n_bins in (64, 100, 256, 4096):
        got = proposal.n_valid(geo, n_bins)
        for g, v in zip(geo, got):
            I = g[4]
            width = max(1, (I + n_bins - 1) // n_bins)
            assert v == len({i // width for i in range(I)})
            assert v <= n_bins


def test_packed_batch_generator_matches_the_list_form():
    """make_batch_csr packs exactly the curves make_batch_workload makes (same seed)."""
    import synth
    ws = synth.make_batch_workload(n_curves=5, seed=77, planet_frac=0.5, with_periods=False)
    off, t, f, e, planets = synth.make_batch_csr((5, 77, 0.5))
    assert off.tolist() == [0] + np.cumsum([w.time.size for w in ws]).tolist()
    for c, w in enumerate(ws):
        np.testing.assert_array_equal(t[off[c]:off[c + 1]], w.time)
        np.testing.assert_array_equal(f[off[c]:off[c + 1]], w.flux)
        np.testing.assert_array_equal(e[off[c]:off[c + 1]], w.flux_err)
        assert planets[c] == w.planets
