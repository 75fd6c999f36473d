"""The allocation-free periodic entry point (cetra_periodic_device_static).

It exists for callers that cannot allocate device memory while they run (a
fixed memory pool, buffers handed in by a host application, a workspace sized
once for the linear grid): its scratch lives in a static device array of the
library. Here it is called through the C ABI and must reproduce the ordinary
cetra_periodic_device on two calls in a row with different period grids (the
second call finds the first call's scratch contents and must not depend on
them). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _outputs(torch, K, dev):
    out = {k: torch.empty(K, dtype=torch.float64, device=dev)
           for k in ("dlogl", "t0", "duration", "depth", "depth_var")}
    out["i"] = torch.empty(K, dtype=torch.int64, device=dev)
    out["j"] = torch.empty(K, dtype=torch.int32, device=dev)
    return out


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_scratch_entry_point_matches_ordinary_one():
    import torch
    import synth
    from synth.lightcurves import custom, HOUR
    from paper_2503_20875_gb300 import (Context, Plan, cetra_resample_device, cetra_linear_device,
                                        cetra_periodic_device)
    from paper_2503_20875_gb300 import _native as N

    w = custom(seed=21, n_points=6000, cadence_s=120.0, durations_h=(0.5, 1.0, 2.0, 4.0),
               planets=[dict(P=1.9, t0=0.4, D=2.0 * HOUR, depth=2e-3, b=0.3)])
    grids = [synth.log_grid(0.5, 4.0, 300), synth.log_grid(0.45, 6.5, 517)]
    dev = torch.device("cuda", 0)
    ctx = Context(0)
    plan = Plan(ctx, w.time, w.flux, w.flux_err, w.durations, w.template, cadence=w.cadence,
                t0_step=w.t0_step)
    kmax = max(g.size for g in grids)
    ws = torch.empty(plan.workspace_bytes(kmax), dtype=torch.uint8, device=dev)
    grid_bytes = plan.workspace_bytes(0)
    d = [torch.as_tensor(a, device=dev) for a in (w.time, w.flux, w.flux_err)]
    cetra_resample_device(ctx, plan, *d, ws)
    cetra_linear_device(ctx, plan, ws)
    for periods in grids:
        K = periods.size
        d_P = torch.as_tensor(periods, device=dev)
        ref = _outputs(torch, K, dev)
        cetra_periodic_device(ctx, plan, ws, d_P, None, ref)
        got = _outputs(torch, K, dev)
        rc = N.lib.cetra_periodic_device_static(
            ctx.handle, plan.handle, _ptr(ws), grid_bytes, _ptr(d_P), K, None,
            _ptr(got["dlogl"]), _ptr(got["t0"]), _ptr(got["duration"]), _ptr(got["depth"]),
            _ptr(got["depth_var"]), _ptr(got["i"]), _ptr(got["j"]))
        assert rc == N.CETRA_OK, N.lib.cetra_last_error(ctx.handle)
        torch.cuda.synchronize()
        r = {k: v.cpu().numpy() for k, v in ref.items()}
        g = {k: v.cpu().numpy() for k, v in got.items()}
        np.testing.assert_array_equal(g["i"], r["i"])
        np.testing.assert_array_equal(g["j"], r["j"])
        assert not np.isnan(r["dlogl"]).any()
        for k in ("dlogl", "t0", "duration", "depth", "depth_var"):
            np.testing.assert_allclose(g[k], r[k], rtol=1e-6, atol=0)

    # sizes beyond the static array are refused before any device work
    big = N.CETRA_STATIC_MAX_PERIODS + 1 if hasattr(N, "CETRA_STATIC_MAX_PERIODS") else 262145
    rc = N.lib.cetra_periodic_device_static(ctx.handle, plan.handle, _ptr(ws), grid_bytes,
                                            _ptr(ws), big, None, None, None, None, None, None,
                                            None, None)
    assert rc == N.CETRA_ECAPACITY
    assert b"static scratch limit" in N.lib.cetra_last_error(ctx.handle)
