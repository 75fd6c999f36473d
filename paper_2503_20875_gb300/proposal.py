"""Learned period-interval proposal for the batched search (not in the paper).

The periodic search (Sec. 2.3) folds every trial period; this aid picks, per curve, a small
fraction of log-spaced period intervals to fold instead:
  1. cetra_batch_features: every window's LR (positive depths), max-pooled to
     [durations][n_bins] per curve.
  2. cetra_cnn_forward: per-bin probability that a bin holds a transit; cetra_cnn_map: that
     probability times the bin's best window LR.
  3. cetra_cnn_comb: a score for each period interval from that map.
  4. cetra_batch_run_proposed: each curve's best intervals -> the fold work items (8-period
     groups) of their periods, chosen on the device, and the fold over those periods only.
The network is trained on injection curves: the labels mark the bins that hold an injected
transit (its mid-time +- half its duration). Every step of the arithmetic runs in the
library's kernels; this module only does the bookkeeping on the host.
"""
from __future__ import annotations

import math

import numpy as np

from .api import Batch, CNN, Context, cetra_cnn_comb, cetra_cnn_map

N_BINS = 4096
N_INTERVALS = 512
P_LO = 0.5


# --------------------------------------------------------------------------- host bookkeeping

def geometry(batch: Batch):
    """Per curve: (t_ref, period_min, ratio, n_periods, n_t0, first_item)."""
    return [batch.curve(c) for c in range(batch.n)]


def t0_index(t, t_ref, info):
    """Position of time t on a curve's t0 grid: t0_i = t_ref + (i p / q - n_pad) cadence."""
    return (t - t_ref) / info["t0_step"] + info["n_pad"] * info["q"] / info["p"]


def labels(geo, info, planets_per_curve, n_bins=N_BINS):
    """[n_curves][n_bins] float32: 1 for the bins of each curve's t0 grid that hold an
    injected transit (any t0 within D/2 of a transit mid-time), else 0."""
    out = np.zeros((len(geo), n_bins), np.float32)
    s = info["t0_step"]
    for idx, (g, planets) in enumerate(zip(geo, planets_per_curve)):
        t_ref, I = g[0], g[4]
        if I <= 0 or not planets:
            continue
        width = (I + n_bins - 1) // n_bins
        t_first = t_ref - info["n_pad"] * info["cadence"]  # time of t0 cell 0
        t_last = t_first + (I - 1) * s
        diff = np.zeros(n_bins + 1, np.int64)
        for pl in planets:
            P, t0, D = pl["P"], pl["t0"], pl["D"]
            # mid-times t0 + n P whose +-D/2 span meets the grid (cells 0 .. I - 1)
            n = np.arange(math.floor((t_first - 0.5 * D - t0) / P),
                          math.ceil((t_last + 0.5 * D - t0) / P) + 1)
            ic = t0_index(t0 + n * P, t_ref, info)
            hw = 0.5 * D / s
            lo = np.maximum(np.ceil(ic - hw), 0).astype(np.int64)
            hi = np.minimum(np.floor(ic + hw), I - 1).astype(np.int64)
            ok = lo <= hi
            np.add.at(diff, lo[ok] // width, 1)
            np.add.at(diff, hi[ok] // width + 1, -1)
        out[idx] = (np.cumsum(diff[:n_bins]) > 0).astype(np.float32)
    return out


def n_valid(geo, n_bins=N_BINS):
    """Number of feature bins that hold t0 cells, per curve: ceil(I / ceil(I / n_bins))."""
    out = []
    for g in geo:
        I = g[4]
        out.append(0 if I <= 0 else -(-I // ((I + n_bins - 1) // n_bins)))
    return np.array(out, np.int32)


def bin_days(geo, info, n_bins=N_BINS):
    """Width in days of one feature bin of each curve (0 for a curve without t0 cells)."""
    s = info["t0_step"]
    return np.array([((g[4] + n_bins - 1) // n_bins) * s if g[4] > 0 else 0.0 for g in geo],
                    np.float64)


def period_max(geo):
    """Upper edge for the intervals: just above the longest trial period of the batch."""
    top = [g[1] * g[2] ** (g[3] - 1) for g in geo if g[3] > 0]
    return max(top) * (1.0 + 1e-9) if top else 2.0 * P_LO


# --------------------------------------------------------------------------- device steps

def train(cnn: CNN, d_features, d_labels, epochs=3, batch_size=32, lr=2e-3, pos_weight=20.0,
          seed=0):
    """Adam over mini-batches of curves; returns the mean loss of each epoch."""
    n = d_features.shape[0]
    rng = np.random.default_rng(seed)
    history = []
    for _ in range(epochs):
        losses = []
        for blk in rng.permutation(n // batch_size):
            a, b = blk * batch_size, (blk + 1) * batch_size
            losses.append(cnn.backward(d_features[a:b], d_labels[a:b], pos_weight))
            cnn.adam(lr)
        history.append(float(np.mean(losses)))
    return history


def predict(cnn: CNN, d_features, chunk=None):
    """Per-bin transit probabilities [n_curves][n_bins] (torch CUDA tensor)."""
    import torch
    n = d_features.shape[0]
    chunk = chunk or cnn.max_batch
    out = torch.empty((n, d_features.shape[2]), dtype=torch.float32, device=d_features.device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        cnn.forward(d_features[a:b], out[a:b])
    return out


def learned_map(ctx: Context, cnn: CNN, d_features):
    """Transit probability x best window LR per bin (torch CUDA tensor [n_curves][n_bins])."""
    import torch
    prob = predict(cnn, d_features)
    out = torch.empty_like(prob)
    cetra_cnn_map(ctx, prob, d_features, out)
    return out


def lr_map(ctx: Context, d_features):
    """The map without the network: each bin's best window LR (probability 1 everywhere)."""
    import torch
    ones = torch.ones((d_features.shape[0], d_features.shape[2]), dtype=torch.float32,
                      device=d_features.device)
    out = torch.empty_like(ones)
    cetra_cnn_map(ctx, ones, d_features, out)
    return out


def interval_scores(ctx: Context, geo, info, d_map, p_hi, n_intervals=N_INTERVALS):
    """Comb scores [n_curves][n_intervals] of per-bin maps d_map (torch CUDA tensor)."""
    import torch
    dev = d_map.device
    T = d_map.shape[1]
    bw = torch.as_tensor(bin_days(geo, info, T), device=dev)
    nv = torch.as_tensor(n_valid(geo, T), device=dev)
    scores = torch.empty((d_map.shape[0], n_intervals), dtype=torch.float32, device=dev)
    cetra_cnn_comb(ctx, d_map.contiguous(), bw, P_LO, p_hi, n_intervals, scores, nv)
    return scores


def propose_and_fold(ctx: Context, batch: Batch, d_map, p_hi, top_frac=0.05,
                     n_intervals=N_INTERVALS, geo=None):
    """Comb the maps and fold each curve's best intervals (selection on the device).
    Returns (best dict, n_items, n_periods). The batch's linear stage must be current
    (cetra_batch_features ran on it)."""
    geo = geo if geo is not None else geometry(batch)
    scores = interval_scores(ctx, geo, batch.info, d_map, p_hi, n_intervals)
    return batch.run_proposed(scores, P_LO, p_hi, top_frac)
