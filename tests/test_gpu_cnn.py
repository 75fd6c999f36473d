"""The learned period-interval proposal on the GPU: the network's forward pass, gradients and
Adam step against the FP64 reference in oracle/cnn.py, the comb against its plain-loop
definition, the batch features and item-list fold against the search oracle, and what the
trained network gains over folding a random or an untrained choice of intervals."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu

CAD = 1800.0 / 86400.0
STEP = 600.0 / 86400.0


def _torch():
    import torch
    return torch


def _net(cin, T, B, seed, scale=0.25):
    from paper_2503_20875_gb300 import Context, CNN
    ctx = Context(0)
    net = CNN(ctx, cin, n_bins=T, max_batch=B, seed=seed)
    rng = np.random.default_rng(seed)
    p = np.zeros(net.n_params, np.float32)
    off = 0
    for o, i in ocnn.shapes(cin):
        nw = o * i * ocnn.K
        p[off:off + nw] = rng.normal(0.0, scale, nw)
        p[off + nw:off + nw + o] = rng.normal(0.0, 0.05, o)
        off += nw + o
    net.set_params(p)
    return ctx, net, p


def _inputs(B, cin, T, seed):
    rng = np.random.default_rng(seed)
    f = rng.exponential(4.0, size=(B, cin, T)).astype(np.float32)
    f[rng.uniform(size=f.shape) < 0.1] = 0.0
    y = np.zeros((B, T), np.float32)
    for b in range(B):
        for c in rng.integers(0, T, 6):
            y[b, max(0, c - 5):c + 5] = 1.0
    return f, y


def _layer_slices(cin):
    out, off = [], 0
    for o, i in ocnn.shapes(cin):
        out.append(slice(off, off + o * i * ocnn.K + o))
        off += o * i * ocnn.K + o
    return out


@pytest.mark.parametrize("cin,T,B", [(16, 512, 3), (1, 256, 2), (32, 768, 1), (16, 4096, 2)])
def test_forward_matches_oracle(cin, T, B):
    """Probabilities within 2e-5: FP32 sums of at most 288 BF16 x FP32 products per layer
    (relative error ~ 288 u_32 of the sum of magnitudes, ~2e-5 of a logit of order 1, and
    the sigmoid's slope is <= 1/4)."""
    torch = _torch()
    ctx, net, p = _net(cin, T, B, seed=cin + T)
    f, _ = _inputs(B, cin, T, seed=1)
    d_f = torch.from_numpy(f).cuda()
    d_p = torch.empty((B, T), dtype=torch.float32, device="cuda")
    net.forward(d_f, d_p)
    ref = ocnn.probabilities(p, f)
    np.testing.assert_allclose(d_p.cpu().numpy(), ref, rtol=0, atol=2e-5)


@pytest.mark.parametrize("cin,T,B", [(16, 512, 3), (4, 256, 2), (16, 4096, 2)])
def test_gradients_match_oracle(cin, T, B):
    """Loss to 1e-5 (relative) and every layer's gradient to 2e-3 of that layer's largest
    component (FP32 forward and backward sums; a ReLU whose input is within rounding of 0
    may switch between the two sides, which moves a few components by that much)."""
    torch = _torch()
    ctx, net, p = _net(cin, T, B, seed=7 + cin)
    f, y = _inputs(B, cin, T, seed=2)
    loss, g = net.backward(torch.from_numpy(f).cuda(), torch.from_numpy(y).cuda(), 8.0,
                           grads=True)
    ref_loss, ref_g = ocnn.loss_and_grads(p, f, y, 8.0)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    for sl in _layer_slices(cin):
        scale = np.abs(ref_g[sl]).max()
        np.testing.assert_allclose(g[sl], ref_g[sl], rtol=0, atol=2e-3 * scale)


def test_adam_steps_match_oracle():
    """Two Adam steps on two different batches: the parameters follow the FP64 reference
    (its own gradients and moments) to 2 % of the learning rate, except where a gradient is
    within the gradient tolerance (2e-3 of its layer's largest) of 0: there the direction of
    the step is not fixed by the arithmetic."""
    torch = _torch()
    cin, T, B, lr = 8, 256, 2, 1e-3
    ctx, net, p0 = _net(cin, T, B, seed=11)
    p_ref, m, v = p0.astype(np.float64), np.zeros(p0.size), np.zeros(p0.size)
    small = np.zeros(p0.size, bool)
    for step in (1, 2):
        f, y = _inputs(B, cin, T, seed=20 + step)
        net.backward(torch.from_numpy(f).cuda(), torch.from_numpy(y).cuda(), 5.0)
        net.adam(lr)
        _, g = ocnn.loss_and_grads(p_ref.astype(np.float32), f, y, 5.0)
        for sl in _layer_slices(cin):
            small[sl] |= np.abs(g[sl]) <= 2e-3 * np.abs(g[sl]).max()
        p_ref, m, v = ocnn.adam_step(p_ref, g, m, v, step, lr)
    got = net.get_params()
    assert (~small).mean() > 0.6
    np.testing.assert_allclose(got[~small], p_ref[~small], rtol=0, atol=0.02 * lr)
    assert np.all(np.abs(got - p0) <= 2 * lr * 1.001 + 1e-7)


def test_comb_matches_oracle():
    """Comb scores against the plain-loop definition (same FP64 trial periods, exact
    integer epochs): FP32 sums of at most a few hundred terms in [0, 1]."""
    torch = _torch()
    from paper_2503_20875_gb300 import Context, cetra_cnn_comb
    ctx = Context(0)
    rng = np.random.default_rng(5)
    T, n = 256, 24
    prob = rng.uniform(size=(5, T)).astype(np.float32) ** 4
    prob[1, 3::37] = 1.0
    bw = np.array([0.01, 0.02, 0.0, 0.013, 0.011])
    nv = np.array([256, 200, 256, 97, 0], np.int32)
    for valid in (None, nv):
        scores = torch.empty((5, n), dtype=torch.float32, device="cuda")
        cetra_cnn_comb(ctx, torch.from_numpy(prob).cuda(), torch.from_numpy(bw).cuda(), 0.3, 1.9,
                       n, scores, None if valid is None else torch.from_numpy(valid).cuda())
        ref = ocnn.comb(prob, bw, 0.3, 1.9, n, valid)
        got = scores.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=2e-6, atol=1e-7)
        assert np.all(got[2] == 0.0)
    assert np.all(got[4] == 0.0)


def test_comb_full_width_matches_oracle():
    """The comb at the full 4,096-bin width on a learned-map-like input (sparse positive
    bins), over narrow intervals at short and long periods (cheap for the plain loops)."""
    torch = _torch()
    from paper_2503_20875_gb300 import Context, cetra_cnn_comb
    ctx = Context(0)
    rng = np.random.default_rng(12)
    T = 4096
    m = (rng.uniform(size=(2, T)) ** 8).astype(np.float32)
    m[0, 100::731] += 3.0  # a pulse train every 731 bins
    bw = np.array([0.1, 0.013])
    nv = np.array([4096, 3500], np.int32)
    for lo, hi, n in ((0.5, 0.5 * 1.004 ** 3, 3), (73.0, 73.3, 2), (150.0, 162.0, 2)):
        scores = torch.empty((2, n), dtype=torch.float32, device="cuda")
        cetra_cnn_comb(ctx, torch.from_numpy(m).cuda(), torch.from_numpy(bw).cuda(), lo, hi, n,
                       scores, torch.from_numpy(nv).cuda())
        ref = ocnn.comb(m, bw, lo, hi, n, nv)
        np.testing.assert_allclose(scores.cpu().numpy(), ref, rtol=5e-6, atol=1e-6)


def test_comb_large_map_from_global_memory():
    """A map too large for shared memory (32,768 bins) is read from global memory."""
    torch = _torch()
    from paper_2503_20875_gb300 import Context, cetra_cnn_comb
    ctx = Context(0)
    T = 32768
    m = np.zeros((1, T), np.float32)
    m[0, 11::1000] = 1.0  # 33 pulses every 1000 bins
    scores = torch.empty((1, 8), dtype=torch.float32, device="cuda")
    cetra_cnn_comb(ctx, torch.from_numpy(m).cuda(), torch.tensor([1.0], dtype=torch.float64,
                   device="cuda"), 600.0, 1500.0, 8, scores)
    got = scores.cpu().numpy()[0]
    q = int(math.floor(8 * math.log(1000.0 / 600.0) / math.log(1500.0 / 600.0)))
    assert got[q] == pytest.approx(math.sqrt(33.0), rel=1e-6)
    assert np.argmax(got) == q


def test_proposal_map_matches_oracle():
    torch = _torch()
    from paper_2503_20875_gb300 import Context, cetra_cnn_map
    ctx = Context(0)
    rng = np.random.default_rng(6)
    f = (rng.normal(size=(3, 5, 300)) * 10).astype(np.float32)
    p = rng.uniform(size=(3, 300)).astype(np.float32)
    out = torch.empty((3, 300), dtype=torch.float32, device="cuda")
    cetra_cnn_map(ctx, torch.from_numpy(p).cuda(), torch.from_numpy(f).cuda(), out)
    np.testing.assert_allclose(out.cpu().numpy(), ocnn.proposal_map(p, f), rtol=3e-7, atol=0)


def _batch(n, seed, ratio=1.003, **kw):
    from paper_2503_20875_gb300 import Context, Batch
    ws = synth.make_batch_workload(n_curves=n, seed=seed, **kw)
    ctx = Context(0)
    b = Batch(ctx, [(w.time, w.flux, w.flux_err) for w in ws], ws[0].durations, ws[0].template,
              0.5, None, ratio, cadence=CAD, t0_step=STEP)
    return ctx, b, ws


def test_batch_features_match_oracle():
    """Max-pooled LR of the dimming windows, from the oracle's per-window depth and LR. A
    bin's maximum moves by at most the largest per-window LR bound of the linear parity
    tests in that bin; a window whose depth is within its bound of 0 may count on one side
    only, which its own LR (then tiny) covers."""
    from tests._parity import linear_bounds, window_lengths
    ctx, b, ws = _batch(3, seed=31, max_sectors=2)
    n_bins = 512
    feats = b.features(n_bins).cpu().numpy()
    for c, w in enumerate(ws):
        r = oracle.search(w.time, w.flux, w.flux_err, w.durations, w.template, None,
                          cadence=CAD, t0_step=STEP, with_kappa=True)
        I = b.curve(c)[4]
        assert r["dlogl"].shape == (w.durations.size, I)
        ok = np.isfinite(r["dlogl"])
        d, v, l, kap = (np.where(ok, r[k], 1.0) for k in ("depth", "depth_var", "dlogl", "kappa"))
        n_w = np.broadcast_to(window_lengths(r["geom"], w.durations)[:, None], d.shape)
        b_d, _, b_l = linear_bounds(d, v, l, kap, n_w, 1e-6)
        lr = np.where(ok & (d > 0), l, 0.0)
        slack = np.where(ok, b_l + np.where(np.abs(d) <= b_d, l, 0.0), 0.0)
        width = (I + n_bins - 1) // n_bins
        ref, tol = np.zeros((w.durations.size, n_bins)), np.zeros((w.durations.size, n_bins))
        for k in range(n_bins):
            if k * width < I:
                sl = slice(k * width, min(I, (k + 1) * width))
                ref[:, k] = lr[:, sl].max(axis=1)
                tol[:, k] = slack[:, sl].max(axis=1)
        err = np.abs(feats[c].astype(np.float64) - ref)
        assert np.all(err <= tol + 1e-7 * ref), float(np.max(err - tol))


def test_run_items_matches_oracle_on_the_chosen_periods():
    """Folding a subset of 8-period groups gives, per curve, the oracle's best model over
    exactly those periods; all groups give the full run."""
    from paper_2503_20875_gb300.api import batch_period_grid
    ctx, b, ws = _batch(4, seed=32, max_sectors=2)
    full = b.run()
    geo = [b.curve(c) for c in range(b.n)]
    rng = np.random.default_rng(3)
    items, chosen = [], []
    for c, g in enumerate(geo):
        n_groups = math.ceil(g[3] / 8)
        sel = np.sort(rng.choice(n_groups, size=max(1, n_groups // 10), replace=False))
        items.append(g[5] + sel)
        chosen.append(sel)
    got = b.run_items(np.concatenate(items), linear=True)
    for c, (g, w) in enumerate(zip(geo, ws)):
        P = batch_period_grid(g[1], g[2], g[3])
        ks = np.concatenate([np.arange(8 * x, min(g[3], 8 * x + 8)) for x in chosen[c]])
        r = oracle.search(w.time, w.flux, w.flux_err, w.durations, w.template, P[ks],
                          cadence=CAD, t0_step=STEP)
        per = r["periodic"]["dlogl"]
        kb = int(np.nanargmax(per))
        assert got["dlogl"][c] == pytest.approx(per[kb], rel=1e-5)
        assert got["dlogl"][c] <= full["dlogl"][c]
        if got["k"][c] != ks[kb]:  # an epsilon-tie between periods: the GPU's pick is as good
            j = list(ks).index(got["k"][c])
            assert per[kb] - per[j] <= 1e-5 * per[kb]
    every = np.concatenate([g[5] + np.arange(math.ceil(g[3] / 8)) for g in geo])
    all_items = b.run_items(every, linear=False)
    for key in ("k", "i", "j", "dlogl"):
        np.testing.assert_array_equal(all_items[key], full[key])


def test_run_proposed_matches_oracle_selection():
    """The device-side choice of work items equals the plain definition in oracle/cnn.py on
    the same scores (exact integers), and its fold equals folding those items."""
    torch = _torch()
    ctx, b, ws = _batch(6, seed=33, max_sectors=3, ratio=None)
    b.features(512)  # resample + linear stage
    geo = [b.curve(c) for c in range(b.n)]
    curves = []
    for g, w in zip(geo, ws):
        T = w.time.max() - w.time.min()
        P = oracle.period_grid(g[1], g[2], 0.5 * T)
        assert P.size == g[3]
        curves.append((P, g[5]))
    p_hi = max(P[-1] for P, _ in curves) * 1.001
    rng = np.random.default_rng(8)
    for n_int, frac in ((512, 0.05), (64, 0.3), (1024, 0.01), (16, 1.0)):
        sc = rng.uniform(size=(b.n, n_int)).astype(np.float32)
        sc[0, :5] = np.nan
        sc[1, :] = 0.5  # all tied: the lowest intervals win
        best, n_it, n_per, items = b.run_proposed(torch.from_numpy(sc).cuda(), 0.5, p_hi, frac,
                                                  items=True)
        ref, ref_per = ocnn.propose_items(curves, sc, 0.5, p_hi, frac)
        np.testing.assert_array_equal(items, ref)
        assert n_it == ref.size and n_per == ref_per
        again = b.run_items(items, linear=False)
        for key in ("k", "i", "j", "dlogl"):
            np.testing.assert_array_equal(best[key], again[key])
    # a narrow proposal range: periods outside [p_lo, p_hi) are never folded
    sc = np.ones((b.n, 8), np.float32)
    _, _, n_per, items = b.run_proposed(torch.from_numpy(sc).cuda(), 2.0, 3.0, 1.0, items=True)
    ref, ref_per = ocnn.propose_items(curves, sc, 2.0, 3.0, 1.0)
    np.testing.assert_array_equal(items, ref)
    assert n_per == ref_per
    from paper_2503_20875_gb300 import CetraError
    with pytest.raises(CetraError):
        b.run_proposed(torch.from_numpy(sc).cuda(), 2.0, 1.0, 0.5)
    with pytest.raises(CetraError):
        b.run_proposed(torch.from_numpy(sc).cuda(), 0.5, 3.0, 0.0)


def test_search_proposed_one_call_equals_the_steps():
    """cetra_batch_search_proposed gives the same best models and fold work as the step by
    step proposal (features, network, map, comb, device selection and fold)."""
    torch = _torch()
    from paper_2503_20875_gb300 import CNN, proposal
    ctx, b, ws = _batch(20, seed=34, max_sectors=4, ratio=None)
    net = CNN(ctx, b.info["n_dur"], n_bins=1024, max_batch=8, seed=5)
    geo = proposal.geometry(b)
    p_hi = proposal.period_max(geo)
    one, n_it1, n_per1 = b.search_proposed(net, n_intervals=128, p_lo=0.5, p_hi=p_hi,
                                           top_frac=0.1)
    feats = b.features(1024)
    m = proposal.learned_map(ctx, net, feats)
    steps, n_it2, n_per2 = proposal.propose_and_fold(ctx, b, m, p_hi, 0.1, n_intervals=128,
                                                     geo=geo)
    assert (n_it1, n_per1) == (n_it2, n_per2)
    for key in ("k", "i", "j", "dlogl", "period", "t0"):
        np.testing.assert_array_equal(one[key], steps[key])
    # default upper edge (p_hi <= 0) runs too
    b.search_proposed(net, n_intervals=64, top_frac=0.2)


def _recovered(period, planets):
    if not planets or not np.isfinite(period):
        return False
    Pt = planets[0]["P"]
    return any(abs(period - m * Pt) <= 0.01 * m * Pt for m in (0.5, 1.0, 2.0))


def test_learned_proposal_gain():
    """Train on injection curves, then fold only each curve's best 5 % of period intervals.

    The map the comb reads is the trained network's transit probability times each bin's best
    window LR. Against the same comb over the LR alone (the method without the network), over
    the untrained network's map, and against a random choice of intervals of the same size,
    the trained map must recover clearly more of the injected planets, near the full search,
    while folding a small fraction of the trial periods. Curves of 1-13 sectors, where single
    transits are weak and the window LR alone is a poor guide."""
    torch = _torch()
    from paper_2503_20875_gb300 import CNN, proposal
    n_bins, frac = 4096, 0.05
    # training set: every curve carries a planet
    ctx, tb, tws = _batch(1024, seed=41, max_sectors=13, planet_frac=1.0, snr_range=(6.0, 20.0),
                          ratio=None)
    d_f = tb.features(n_bins)
    lab = proposal.labels(proposal.geometry(tb), tb.info, [w.planets for w in tws], n_bins)
    d_y = torch.from_numpy(lab).cuda()
    tb.close()
    net = CNN(ctx, d_f.shape[1], n_bins=n_bins, max_batch=32, seed=3)
    untrained = CNN(ctx, d_f.shape[1], n_bins=n_bins, max_batch=32, seed=3)
    hist = proposal.train(net, d_f, d_y, epochs=8, batch_size=32, lr=2e-3, pos_weight=20.0)
    assert hist[-1] < 0.92 * hist[0]  # the loss falls (transits of long curves are hard to mark)
    del d_f
    # evaluation set (other seeds), the per-curve period grids of the batched form
    _, eb, ews = _batch(128, seed=42, max_sectors=13, planet_frac=1.0, snr_range=(6.0, 20.0),
                        ratio=None)
    geo = proposal.geometry(eb)
    p_hi = proposal.period_max(geo)
    full = eb.run()
    e_f = eb.features(n_bins)
    maps = {"learned": proposal.learned_map(ctx, net, e_f),
            "lr_only": proposal.lr_map(ctx, e_f),
            "untrained": proposal.learned_map(ctx, untrained, e_f)}
    res = {}
    for name, m in maps.items():
        best, n_it, n_per = proposal.propose_and_fold(ctx, eb, m, p_hi, frac, geo=geo)
        res[name] = (sum(_recovered(p, w.planets) for p, w in zip(best["period"], ews)), n_per)
        if name == "learned":  # the fold over the chosen periods never beats the full search
            assert np.all(best["dlogl"] <= full["dlogl"])
    rnd = torch.rand((eb.n, proposal.N_INTERVALS), generator=torch.Generator().manual_seed(5))
    best, _, n_per = eb.run_proposed(rnd.cuda(), proposal.P_LO, p_hi, frac)
    res["random"] = (sum(_recovered(p, w.planets) for p, w in zip(best["period"], ews)), n_per)
    n_full = sum(_recovered(p, w.planets) for p, w in zip(full["period"], ews))
    total = sum(g[3] for g in geo)
    print(f"full search {n_full}/{len(ews)}; " + "; ".join(
        f"{k} {v[0]}/{len(ews)} folding {v[1] / total:.3f} of the periods"
        for k, v in res.items()))
    n = len(ews)
    assert res["learned"][1] <= 0.1 * total
    assert res["learned"][0] >= res["lr_only"][0] + 0.1 * n
    assert res["learned"][0] >= res["untrained"][0] + 0.05 * n
    assert res["learned"][0] >= res["random"][0] + 0.2 * n
    assert res["learned"][0] >= 0.75 * n_full
