"""Run the CUDA path and the FP64 oracle on the same inputs and compare them.

Tolerances (FP32 kernels against the FP64 oracle):
  linear, every non-null cell: with A = depth/var, B = 1/var, kappa = sum |m W y|
  (oracle), window length n_w and u = 2^-24,
      tau_A = r |A| + (n_w + 4) u kappa,    tau_B = (r + (n_w + 4) u) B
      |depth - depth_o| <= (tau_A + |depth_o| tau_B) / B + u |depth_o|
      |LR - LR_o|       <= |depth_o| tau_A + LR_o tau_B / B + u LR_o
  This is the worst-case bound of a length-n_w FP32 dot product plus input
  rounding; cancellation in A (LR near 0) is what the kappa term covers.
  linear, cells with LR_o >= 25 (the cells that matter for detection):
      |LR - LR_o| <= r_flat LR_o
  periodic, per period: the argmax (i, j) is identical, unless the oracle's
  own LR at the GPU's argmax is within r_flat of the oracle's maximum (an
  epsilon-tie between windows, reported); LR, depth and var_Z within r_flat
  relative where LR_o >= 25 and within r_low below that (r_low = r_flat by
  default: the flat bound holds at every per-period winner); t0 and duration
  exact at identical indices.
Null cells and null periods must coincide exactly.
"""
from __future__ import annotations

import numpy as np

import oracle

U = 2.0 ** -24


def gpu_search(time, flux, flux_err, durations, tmpl, periods=None, mask=None, L=1024, **params):
    import torch
    from paper_2503_20875_gb300 import Context, Plan, DeviceSearch
    ctx = Context(0)
    plan = Plan(ctx, time, flux, flux_err, durations, tmpl, template_samples=L, **params)
    P = np.asarray(periods if periods is not None else [], np.float64)
    ds = DeviceSearch(ctx, plan, P, mask)
    dev = torch.device("cuda", 0)
    d_t = torch.as_tensor(np.ascontiguousarray(time, np.float64), device=dev)
    d_f = torch.as_tensor(np.ascontiguousarray(flux, np.float32), device=dev)
    d_e = torch.as_tensor(np.ascontiguousarray(flux_err, np.float32), device=dev)
    ds.run(d_t, d_f, d_e, periodic=P.size > 0, logl0=True)
    torch.cuda.synchronize()
    out = {"info": plan.info, "depth": ds.depth.cpu().numpy(), "depth_var": ds.depth_var.cpu().numpy(),
           "dlogl": ds.dlogl.cpu().numpy(), "logl0": float(ds.logl0.cpu()[0]),
           "launches": ctx.launches}
    if P.size:
        out["periodic"] = {k: v.cpu().numpy() for k, v in ds.out.items()}
    del ds, plan, ctx
    return out


def oracle_search(time, flux, flux_err, durations, tmpl, periods=None, mask=None, L=1024,
                  cadence=0.0, t0_step=0.0, flux_is_offset=False):
    return oracle.search(time, flux, flux_err, durations, tmpl, periods, cadence=cadence,
                         t0_step=t0_step, L=L, flux_is_offset=flux_is_offset, mask=mask,
                         with_kappa=True)


def window_lengths(geom, durations):
    return np.asarray(durations) / geom.cadence + 2.0


def linear_bounds(orc_depth, orc_var, orc_lr, kappa, n_w, r):
    A = orc_depth / orc_var
    B = 1.0 / orc_var
    tau_A = r * np.abs(A) + (n_w + 4) * U * kappa
    tau_B = (r + (n_w + 4) * U) * B
    b_depth = (tau_A + np.abs(orc_depth) * tau_B) / B + U * np.abs(orc_depth)
    b_lr = np.abs(orc_depth) * tau_A + orc_lr * tau_B / B + U * np.abs(orc_lr)
    b_var = tau_B / B ** 2 + U * orc_var
    return b_depth, b_var, b_lr


def compare_linear(gpu, orc, durations, r=1e-6, r_flat=1e-5, lr_sig=25.0, rows=None, cols=None):
    """Element-by-element comparison of the [J][I] linear outputs. ``rows``/``cols``
    select a subset (sampled cells) when the oracle ran only there."""
    g_d, g_v, g_l = gpu["depth"], gpu["depth_var"], gpu["dlogl"]
    if rows is not None:
        g_d, g_v, g_l = g_d[rows, cols], g_v[rows, cols], g_l[rows, cols]
        o_d, o_v, o_l, kap = orc["depth"], orc["depth_var"], orc["dlogl"], orc["kappa"]
        n_w = window_lengths(orc["geom"], np.asarray(durations)[rows])
    else:
        o_d, o_v, o_l, kap = orc["depth"], orc["depth_var"], orc["dlogl"], orc["kappa"]
        n_w = window_lengths(orc["geom"], durations)[:, None]
    null_o = np.isnan(o_l)
    null_g = np.isnan(g_l)
    assert np.array_equal(null_o, null_g), f"null cells differ: {np.sum(null_o != null_g)}"
    ok = ~null_o
    n_w = np.broadcast_to(n_w, o_l.shape)[ok]
    b_d, b_v, b_l = linear_bounds(o_d[ok], o_v[ok], o_l[ok], kap[ok], n_w, r)
    e_d = np.abs(g_d[ok].astype(np.float64) - o_d[ok])
    e_v = np.abs(g_v[ok].astype(np.float64) - o_v[ok])
    e_l = np.abs(g_l[ok].astype(np.float64) - o_l[ok])
    stats = {"cells": int(ok.sum()), "nulls": int(null_o.sum()),
             "max_norm_depth": float(np.max(e_d / b_d, initial=0.0)),
             "max_norm_var": float(np.max(e_v / b_v, initial=0.0)),
             "max_norm_lr": float(np.max(e_l / b_l, initial=0.0))}
    sig = o_l[ok] >= lr_sig
    if sig.any():
        rel = e_l[sig] / o_l[ok][sig]
        stats["sig_cells"] = int(sig.sum())
        stats["max_rel_lr_sig"] = float(rel.max())
        stats["max_rel_depth_sig"] = float((e_d[sig] / np.abs(o_d[ok][sig])).max())
    assert stats["max_norm_depth"] <= 1.0, stats
    assert stats["max_norm_var"] <= 1.0, stats
    assert stats["max_norm_lr"] <= 1.0, stats
    if sig.any():
        assert stats["max_rel_lr_sig"] <= r_flat, stats
    return stats


def compare_periodic(gpu, orc, periods, r_flat=1e-5, r_low=None, lr_sig=25.0, lin=None):
    """Per-period comparison. ``lin`` = (depth, var, lr) oracle arrays used for
    epsilon-tie evaluation (defaults to the oracle's full linear arrays)."""
    if r_low is None:
        r_low = r_flat
    gp, op = gpu["periodic"], orc["periodic"]
    null_o = np.isnan(op["dlogl"])
    null_g = np.isnan(gp["dlogl"])
    assert np.array_equal(null_o, null_g), f"null periods differ: {np.sum(null_o != null_g)}"
    ok = ~null_o
    same = (gp["i"] == op["i"]) & (gp["j"] == op["j"])
    diff = ok & ~same
    ties = 0
    if diff.any():
        dep, var, lr = lin if lin is not None else (orc["depth"], orc["depth_var"], orc["dlogl"])
        k = np.nonzero(diff)[0]
        lr_at, _, _ = oracle.periodic_at(orc["geom"], dep, var, lr, np.asarray(periods)[k],
                                         gp["i"][k], gp["j"][k])
        gap = op["dlogl"][k] - lr_at
        tol = r_flat * np.maximum(op["dlogl"][k], lr_sig)
        bad = ~(gap <= tol)
        assert not bad.any(), {"periods": k[bad][:10].tolist(), "gap": gap[bad][:10].tolist(),
                               "oracle_lr": op["dlogl"][k][bad][:10].tolist()}
        ties = int(diff.sum())
    rel = lambda a, b: np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    m = ok & same
    sig = m & (op["dlogl"] >= lr_sig)
    low = m & (op["dlogl"] < lr_sig)
    stats = {"periods": int(ok.sum()), "null": int(null_o.sum()), "eps_ties": ties,
             "max_rel_lr_sig": float(np.max(rel(gp["dlogl"][sig], op["dlogl"][sig]), initial=0)),
             "max_rel_depth_sig": float(np.max(rel(gp["depth"][sig], op["depth"][sig]), initial=0)),
             "max_rel_var_sig": float(np.max(rel(gp["depth_var"][sig], op["depth_var"][sig]),
                                             initial=0)),
             "max_rel_lr_low": float(np.max(rel(gp["dlogl"][low], op["dlogl"][low]), initial=0)),
             "max_rel_depth_low": float(np.max(rel(gp["depth"][low], op["depth"][low]), initial=0)),
             "max_rel_var_low": float(np.max(rel(gp["depth_var"][low], op["depth_var"][low]),
                                             initial=0))}
    assert stats["max_rel_lr_sig"] <= r_flat, stats
    assert stats["max_rel_depth_sig"] <= r_flat, stats
    assert stats["max_rel_var_sig"] <= r_flat, stats
    assert stats["max_rel_lr_low"] <= r_low, stats
    assert stats["max_rel_depth_low"] <= r_low, stats
    assert stats["max_rel_var_low"] <= r_low, stats
    np.testing.assert_array_equal(gp["duration"][m], op["duration"][m])
    np.testing.assert_allclose(gp["t0"][m], op["t0"][m], rtol=0, atol=1e-9 * max(1.0, np.nanmax(np.abs(op["t0"]))))
    # the global best period
    kg = int(np.nanargmax(gp["dlogl"])) if ok.any() else -1
    ko = int(np.nanargmax(op["dlogl"])) if ok.any() else -1
    if kg != ko:
        assert op["dlogl"][ko] - op["dlogl"][kg] <= r_flat * op["dlogl"][ko], (kg, ko)
    stats["best_k"] = (kg, ko)
    return stats
