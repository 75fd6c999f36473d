"""Pins of the FP64 network reference (oracle/cnn.py) against library routines and
finite differences: it is then the yardstick for the CUDA proposal network."""
import numpy as np
import pytest

from oracle import cnn


def test_conv_is_cross_correlation():
    rng = np.random.default_rng(0)
    from scipy.signal import correlate
    x = rng.normal(size=(1, 1, 50))
    W = rng.normal(size=(1, 1, 9))
    y, _ = cnn.conv(x, W, np.zeros(1))
    ref = correlate(x[0, 0], W[0, 0], mode="same")
    np.testing.assert_allclose(y[0, 0], ref, rtol=1e-12, atol=1e-12)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    w = np.concatenate([rng.normal(size=1000).astype(np.float32),
                        np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5e-3], np.float32)])
    ref = torch.from_numpy(w).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.bf16_round(w), ref)
    assert cnn.bf16_round(np.float32(1 + 2 ** -8)) == 1.0  # a tie goes to even


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    B, cin, T = 2, 3, 40
    f = rng.exponential(3.0, size=(B, cin, T)).astype(np.float32)
    y = (rng.uniform(size=(B, T)) < 0.1).astype(np.float64)
    layers = []
    for o, i in cnn.shapes(cin):
        layers.append((rng.normal(0, 0.4, size=(o, i, cnn.K)), rng.normal(0, 0.1, size=o)))
    loss, flat = cnn.loss_and_grads_layers(layers, f, y, 4.0)
    # central differences on a sample of weights and biases of every layer
    off = 0
    h = 1e-6
    for l, (W, b) in enumerate(layers):
        for idx in list(zip(*[rng.integers(0, s, 4) for s in W.shape])):
            Wp = [(w.copy(), bb.copy()) for w, bb in layers]
            Wm = [(w.copy(), bb.copy()) for w, bb in layers]
            Wp[l][0][idx] += h
            Wm[l][0][idx] -= h
            num = (cnn.loss_and_grads_layers(Wp, f, y, 4.0)[0] -
                   cnn.loss_and_grads_layers(Wm, f, y, 4.0)[0]) / (2 * h)
            ana = flat[off + np.ravel_multi_index(idx, W.shape)]
            assert ana == pytest.approx(num, rel=1e-5, abs=1e-9)
        off += W.size
        for o in range(min(2, b.size)):
            Wp = [(w.copy(), bb.copy()) for w, bb in layers]
            Wm = [(w.copy(), bb.copy()) for w, bb in layers]
            Wp[l][1][o] += h
            Wm[l][1][o] -= h
            num = (cnn.loss_and_grads_layers(Wp, f, y, 4.0)[0] -
                   cnn.loss_and_grads_layers(Wm, f, y, 4.0)[0]) / (2 * h)
            assert flat[off + o] == pytest.approx(num, rel=1e-5, abs=1e-9)
        off += b.size


def test_loss_closed_form():
    """Zero weights and biases: every logit is 0, loss = log 2 (w+ p + 1 - p), p the label rate."""
    rng = np.random.default_rng(3)
    f = rng.exponential(size=(2, 2, 30)).astype(np.float32)
    y = (rng.uniform(size=(2, 30)) < 0.2).astype(np.float64)
    layers = [(np.zeros((o, i, cnn.K)), np.zeros(o)) for o, i in cnn.shapes(2)]
    loss, _ = cnn.loss_and_grads_layers(layers, f, y, 3.0)
    assert loss == pytest.approx(np.log(2) * (3.0 * y.mean() + 1 - y.mean()), rel=1e-12)


def test_adam_matches_torch():
    """Three bias-corrected Adam steps equal torch.optim.Adam's."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(3)]
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step, g in enumerate(grads, 1):
        t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = cnn.adam_step(p, g, m, v, step, 1e-2)
    np.testing.assert_allclose(p, t.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_comb_constant_map_closed_form():
    """A map of ones: every (trial, phase) scores sqrt(E), the largest E at phase 0 of the
    shortest trial of the interval: E = ceil((T 2^32 - 2^31) / F), F = floor(P 2^32 + 1/2)."""
    import math
    T, w, n = 300, 0.1, 12
    sc = cnn.comb(np.ones((1, T)), [w], 0.5, 12.0, n)
    for q in range(n):
        lo = 0.5 * (12.0 / 0.5) ** (q / n) / w
        hi = 0.5 * (12.0 / 0.5) ** ((q + 1) / n) / w
        nP = max(1, math.ceil((hi - lo) * T / lo))
        F = math.floor((lo + (hi - lo) * 0.5 / nP) * 2.0 ** 32 + 0.5)
        E = -(-(T * 2 ** 32 - 2 ** 31) // F)
        assert sc[0, q] == pytest.approx(math.sqrt(E), rel=1e-12)


def test_comb_valid_span_is_a_truncation():
    """Bins past a curve's valid span do not count: the scores equal those of the map cut to
    that span, whatever the bins past it hold."""
    rng = np.random.default_rng(6)
    V, T = 180, 256
    m = rng.uniform(size=(1, T))
    m[0, V:] = 1e6
    a = cnn.comb(m, [0.02], 0.05, 2.0, 10, n_valid=[V])
    b = cnn.comb(m[:, :V], [0.02], 0.05, 2.0, 10)
    np.testing.assert_array_equal(a, b)
    assert a.max() < 1e3


def test_proposal_map_worked_values():
    """p = 0.5 with window LRs 4.5, 8 and -1 in one bin: 0.5 x 8 = 4; zero features give 0."""
    f = np.array([[[4.5, 0.0], [8.0, 0.0], [-1.0, 0.0]]], np.float32)
    got = cnn.proposal_map(np.array([[0.5, 0.9]], np.float32), f)
    np.testing.assert_array_equal(got, [[4.0, 0.0]])


def test_comb_finds_planted_pulse_train():
    """Twenty one-bin pulses every 50 bins from bin 7: the interval holding 50 bins scores
    sqrt(20) (all pulses on one trial), the best of all intervals; the intervals holding the
    half (20 hits of 40 epochs) and the double (10 of 10) score sqrt(10)."""
    import math
    T = 1000
    m = np.zeros((1, T))
    m[0, 7::50] = 1.0
    lo, hi, n = 10.0, 400.0, 64
    sc = cnn.comb(m, [1.0], lo, hi, n)[0]
    qi = int(math.floor(n * math.log(50.0 / lo) / math.log(hi / lo)))
    assert sc[qi] == pytest.approx(math.sqrt(20.0), rel=1e-12)
    assert np.argmax(sc) == qi
    for P in (25.0, 100.0):
        qh = int(math.floor(n * math.log(P / lo) / math.log(hi / lo)))
        assert sc[qh] == pytest.approx(math.sqrt(10.0), rel=1e-12)


def test_comb_null_curve_scores_zero():
    sc = cnn.comb(np.ones((2, 64)), [0.0, -1.0], 0.5, 5.0, 4)
    assert np.all(sc == 0.0)


def test_propose_items_worked_example():
    """Periods 1.0, 1.1, ..., 2.9 (20, first item 7), intervals [1, 1.5), [1.5, 2.25),
    [2.25, 3.375) (p_lo 1, p_hi 3.375, n = 3): periods 0-4 | 5-12 | 13-19. With scores
    (0.2, 0.9, 0.5) and top_frac 0.34, ceil(1.02) = 2 intervals are kept: 1 and 2, i.e.
    periods 5-19, groups 0-2 -> items 7, 8, 9 holding all 20 periods."""
    P = 1.0 + 0.1 * np.arange(20)
    items, n_per = cnn.propose_items([(P, 7)], [[0.2, 0.9, 0.5]], 1.0, 3.375, 0.34)
    np.testing.assert_array_equal(items, [7, 8, 9])
    assert n_per == 20
    # keep one interval: the middle one (periods 5-12) -> groups 0 (k 5-7) and 1 (k 8-12)
    items, n_per = cnn.propose_items([(P, 7)], [[0.2, 0.9, 0.5]], 1.0, 3.375, 0.2)
    np.testing.assert_array_equal(items, [7, 8])
    assert n_per == 16
    # a NaN score ranks lowest; equal scores go to the lower interval
    items, _ = cnn.propose_items([(P, 0)], [[np.nan, 0.5, 0.5]], 1.0, 3.375, 0.2)
    np.testing.assert_array_equal(items, [0, 1])  # interval 1 (k 5-12)


def test_propose_items_everything_and_outside_periods():
    """top_frac = 1 keeps every group holding a period in [p_lo, p_hi); periods outside are
    never chosen; a curve without periods gives nothing."""
    P = np.exp(np.linspace(np.log(0.3), np.log(40.0), 300))
    rng = np.random.default_rng(9)
    sc = rng.uniform(size=(2, 16))
    items, n_per = cnn.propose_items([(P, 0), (np.zeros(0), 38)], sc, 0.5, 20.0, 1.0)
    ok = np.nonzero((P >= 0.5) & (P < 20.0))[0]
    want = np.unique(ok // 8)
    np.testing.assert_array_equal(items, want)
    assert n_per == sum(min(8, 300 - 8 * g) for g in want)


def test_comb_rounds_to_the_nearest_bin_and_stops_at_half_the_span():
    """A pulse train at the nearest bins of a 50.5-bin period (t_e = floor(7 + 50.5 e + 1/2)):
    with V = 1,050 valid bins the single interval [50, 51) has 21 trials whose 11th is exactly
    50.5, which hits all 21 pulses: sqrt(21) (truncating the phases would hit every other one).
    Trials above V/2 are skipped: an interval of periods between V/2 and V scores 0 on a map
    of ones."""
    import math
    V = 1050
    m = np.zeros((1, V))
    e = np.arange(21)
    m[0, np.floor(7 + 50.5 * e + 0.5).astype(int)] = 1.0
    sc = cnn.comb(m, [1.0], 50.0, 51.0, 1)
    assert sc[0, 0] == pytest.approx(math.sqrt(21.0), rel=1e-12)
    ones = np.ones((1, 100))
    assert cnn.comb(ones, [1.0], 55.0, 95.0, 3).max() == 0.0
    assert cnn.comb(ones, [1.0], 30.0, 45.0, 1)[0, 0] > 0.0
    # an interval straddling V/2: the 55-bin period of two pulses (bins 0 and 55) is above
    # V/2 = 50 and skipped; the trials below it catch one pulse of two epochs: 1/sqrt(2)
    two = np.zeros((1, 100))
    two[0, [0, 55]] = 1.0
    assert cnn.comb(two, [1.0], 45.0, 60.0, 1)[0, 0] == pytest.approx(1 / math.sqrt(2), rel=1e-12)
