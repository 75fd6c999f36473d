"""FP64 reference of the period-interval proposal network (test infrastructure only).

Plain definitions, no blocking or fusion, used to check the CUDA forward pass and
gradients on small inputs:
  x0 = log1p(max(features, 0))
  conv(x; W, b)[o, t] = b[o] + sum_i sum_k W[o, i, k] x[i, t + k - 4]   (zero padding)
  layers: conv(in -> 32) ReLU, conv(32 -> 32) ReLU, conv(32 -> 32) ReLU, conv(32 -> 1)
  weights rounded to BF16 (nearest even) before use, biases FP32
  loss = mean over bins of  w+ y softplus(-z) + (1 - y) softplus(z)
Gradients are taken with respect to the rounded weights (what the kernels use).
The flat parameter layout is, per layer, W [out][in][9] then b [out].
"""
from __future__ import annotations

import numpy as np

K = 9
HALF = K // 2
HIDDEN = 32
LAYERS = 4


def bf16_round(w):
    """Round FP32 values to the nearest BF16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(w, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u >> 16) & 1) + 0x7FFF
    u = ((u + r) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def shapes(cin):
    out = []
    for l in range(LAYERS):
        i = cin if l == 0 else HIDDEN
        o = 1 if l == LAYERS - 1 else HIDDEN
        out.append((o, i))
    return out


def unflatten(params, cin):
    p = np.asarray(params, np.float32)
    layers, off = [], 0
    for o, i in shapes(cin):
        W = bf16_round(p[off:off + o * i * K]).reshape(o, i, K)
        off += o * i * K
        b = p[off:off + o].astype(np.float64)
        off += o
        layers.append((W, b))
    assert off == p.size
    return layers


def conv(x, W, b):
    B, cin, T = x.shape
    xp = np.zeros((B, cin, T + 2 * HALF))
    xp[:, :, HALF:HALF + T] = x
    y = np.zeros((B, W.shape[0], T)) + b[None, :, None]
    for k in range(K):
        y += np.einsum("oi,bit->bot", W[:, :, k], xp[:, :, k:k + T])
    return y, xp


def forward(params, features):
    f = np.asarray(features, np.float64)
    return forward_layers(unflatten(params, f.shape[1]), features)


def forward_layers(layers, features):
    f = np.asarray(features, np.float64)
    x = np.log1p(np.maximum(f.astype(np.float32).astype(np.float64), 0.0))
    acts = [x]
    pads = []
    for l, (W, b) in enumerate(layers):
        y, xp = conv(acts[-1], W, b)
        pads.append(xp)
        if l < LAYERS - 1:
            y = np.maximum(y, 0.0)
        acts.append(y)
    return acts, pads, layers


def loss_and_grads(params, features, labels, pos_weight):
    f = np.asarray(features, np.float64)
    return loss_and_grads_layers(unflatten(params, f.shape[1]), features, labels, pos_weight)


def loss_and_grads_layers(layers, features, labels, pos_weight):
    acts, pads, layers = forward_layers(layers, features)
    z = acts[-1][:, 0, :]
    y = np.asarray(labels, np.float64)
    n = z.size
    sp = np.logaddexp(0.0, z)          # softplus(z)
    loss = np.mean(pos_weight * y * (sp - z) + (1 - y) * sp)
    s = 1.0 / (1.0 + np.exp(-z))
    g = ((s * (pos_weight * y + 1 - y) - pos_weight * y) / n)[:, None, :]
    grads = [None] * LAYERS
    for l in range(LAYERS - 1, -1, -1):
        W, b = layers[l]
        if l < LAYERS - 1:
            g = g * (acts[l + 1] > 0)
        xp = pads[l]
        T = g.shape[2]
        dW = np.zeros_like(W)
        for k in range(K):
            dW[:, :, k] = np.einsum("bot,bit->oi", g, xp[:, :, k:k + T])
        db = g.sum(axis=(0, 2))
        grads[l] = (dW, db)
        if l > 0:
            dxp = np.zeros_like(xp)
            for k in range(K):
                dxp[:, :, k:k + T] += np.einsum("oi,bot->bit", W[:, :, k], g)
            g = dxp[:, :, HALF:HALF + T]
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return loss, flat


def probabilities(params, features):
    acts, _, _ = forward(params, features)
    return 1.0 / (1.0 + np.exp(-acts[-1][:, 0, :]))


def adam_step(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step on the FP32 parameters (FP64 arithmetic)."""
    p = np.asarray(params, np.float64)
    g = np.asarray(grads, np.float64)
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return p, m, v


def proposal_map(prob, features):
    """map[b][t] = prob[b][t] max_j max(features[b][j][t], 0): the transit probability times
    the bin's best window likelihood ratio."""
    f = np.maximum(np.asarray(features, np.float32).astype(np.float64), 0.0)
    return np.asarray(prob, np.float32).astype(np.float64) * f.max(axis=1)


def comb(prob, bin_days, p_lo, p_hi, n_intervals, n_valid=None):
    """Period comb over per-bin maps prob [B][T] (bin widths bin_days [B] days), plain loops.

    Curve b has V = n_valid[b] valid bins (all T when n_valid is None). Interval q: edges
    lo = p_lo (p_hi/p_lo)^(q/n), hi = the same at q + 1, in bins blo = lo / w, bhi = hi / w;
    trials Pb_m = blo + (bhi - blo)(m + 1/2) / nP with nP = max(1, ceil((bhi - blo) V / blo)),
    skipped below 1 bin or above V / 2; with F = floor(Pb 2^32 + 1/2), each phase ph < ceil(Pb)
    has the epochs t_e = (ph 2^32 + e F + 2^31) >> 32 < V (exact integers) and scores
    sum_e p[t_e] / sqrt(E). The interval's score is the largest such value, 0 if none is
    positive.
    """
    import math
    prob = np.asarray(prob, np.float64)
    B, T = prob.shape
    out = np.zeros((B, n_intervals))
    for b in range(B):
        w = float(bin_days[b])
        V = T if n_valid is None else min(max(int(n_valid[b]), 0), T)
        if not w > 0.0 or V == 0:
            continue
        for q in range(n_intervals):
            lo = p_lo * (p_hi / p_lo) ** (q / n_intervals)
            hi = p_lo * (p_hi / p_lo) ** ((q + 1) / n_intervals)
            blo, bhi = lo / w, hi / w
            if bhi < 1.0 or blo > 0.5 * V:
                continue
            nP = max(1, math.ceil((bhi - blo) * V / blo))
            best = 0.0
            for m in range(nP):
                Pb = blo + (bhi - blo) * (m + 0.5) / nP
                if Pb < 1.0 or Pb > 0.5 * V:
                    continue
                F = math.floor(Pb * 2.0 ** 32 + 0.5)
                for ph in range(math.ceil(Pb)):
                    idx = []
                    e = 0
                    while True:
                        t = (ph * 2 ** 32 + e * F + 2 ** 31) >> 32
                        if t >= V:
                            break
                        idx.append(t)
                        e += 1
                    best = max(best, prob[b, idx].sum() / math.sqrt(len(idx)))
            out[b, q] = best
    return out


def propose_items(curves, scores, p_lo, p_hi, top_frac):
    """Fold work items a proposal keeps (plain definition).

    curves: per curve (periods, first_item), its trial periods ascending. Interval q spans
    [e_q, e_{q+1}) with e_q = p_lo (p_hi/p_lo)^(q/n); a period outside [p_lo, p_hi) belongs to
    none. Of the intervals holding at least one period, the max(1, ceil(top_frac x their
    number)) with the highest scores are kept (NaN lowest; ties: lower q first); every group
    of 8 consecutive periods (k // 8) holding a period of a kept interval is an item,
    numbered first_item + k // 8. Returns (sorted items, number of periods in them).
    """
    import math
    scores = np.asarray(scores, np.float64)
    n = scores.shape[1]
    edges = np.array([p_lo * (p_hi / p_lo) ** (q / n) for q in range(n + 1)])
    items, n_per = [], 0
    for c, (P, first) in enumerate(curves):
        P = np.asarray(P, np.float64)
        K = P.size
        q = np.searchsorted(edges, P, side="right") - 1
        inside = (q >= 0) & (q < n)
        present = sorted(set(q[inside].tolist()))
        if not present:
            continue
        n_keep = max(1, math.ceil(top_frac * len(present)))

        def rank_key(v):
            s = scores[c, v]
            return (-(s if s == s else -np.inf), v)

        kept = set(sorted(present, key=rank_key)[:n_keep])
        groups = sorted({k // 8 for k in range(K) if inside[k] and q[k] in kept})
        n_per += sum(min(8, K - 8 * g) for g in groups)
        items += [first + g for g in groups]
    return np.array(sorted(items), np.int64), n_per
