"""The allocation-free periodic entry point (cetra_periodic_device_static).

It exists for callers that cannot allocate device memory while they run (a
fixed memory pool, buffers handed in by a host application, a workspace sized
once for the linear grid): its scratch lives in a static device array of the
library. Here it is called through the C ABI and must reproduce the ordinary
cetra_periodic_device on calls in a row with different period grids: a longer
grid, then a shorter one (whose call finds the longer call's keys past its own
last period and must not depend on them), then a grid with a (duration,
period) mask. After each call the static status word reads 0; a wait that gave
up (the bounded-wait self-test, recorded the way a fold records it) reads
CETRA_ETIMEOUT until the next call clears it. This file is collected last on
purpose.
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
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _static_status(N, ctx):
    st = ctypes.c_int(-1)
    rc = N.lib.cetra_static_status(ctx.handle, ctypes.byref(st))
    assert rc == N.CETRA_OK, N.lib.cetra_last_error(ctx.handle)
    return st.value


def test_static_scratch_entry_point_matches_ordinary_one():
    import torch
    import synth
    from synth.lightcurves import custom, HOUR
    from paper_2503_20875_gb300 import (Context, Plan, cetra_resample_device, cetra_linear_device,
                                        cetra_periodic_device)
    from paper_2503_20875_gb300 import _native as N

    w = custom(seed=21, n_points=6000, cadence_s=120.0, durations_h=(0.5, 1.0, 2.0, 4.0),
               planets=[dict(P=1.9, t0=0.4, D=2.0 * HOUR, depth=2e-3, b=0.3)])
    rng = np.random.default_rng(8)
    masked = synth.log_grid(0.5, 5.0, 260)
    mask = (rng.uniform(size=(masked.size, w.durations.size)) < 0.7).astype(np.uint8)
    mask[:9] = 0  # periods with every duration masked are null
    # a longer grid first, then a shorter one, then a masked one
    calls = [(synth.log_grid(0.45, 6.5, 517), None), (synth.log_grid(0.5, 4.0, 300), None),
             (masked, mask)]
    dev = torch.device("cuda", 0)
    ctx = Context(0)
    plan = Plan(ctx, w.time, w.flux, w.flux_err, w.durations, w.template, cadence=w.cadence,
                t0_step=w.t0_step)
    kmax = max(p.size for p, _ in calls)
    ws = torch.empty(plan.workspace_bytes(kmax), dtype=torch.uint8, device=dev)
    grid_bytes = plan.workspace_bytes(0)
    d = [torch.as_tensor(a, device=dev) for a in (w.time, w.flux, w.flux_err)]
    cetra_resample_device(ctx, plan, *d, ws)
    cetra_linear_device(ctx, plan, ws)
    for periods, m in calls:
        K = periods.size
        d_P = torch.as_tensor(periods, device=dev)
        d_m = torch.as_tensor(m, device=dev) if m is not None else None
        ref = _outputs(torch, K, dev)
        cetra_periodic_device(ctx, plan, ws, d_P, d_m, ref)
        got = _outputs(torch, K, dev)
        rc = N.lib.cetra_periodic_device_static(
            ctx.handle, plan.handle, _ptr(ws), grid_bytes, _ptr(d_P), K, _ptr(d_m),
            _ptr(got["dlogl"]), _ptr(got["t0"]), _ptr(got["duration"]), _ptr(got["depth"]),
            _ptr(got["depth_var"]), _ptr(got["i"]), _ptr(got["j"]))
        assert rc == N.CETRA_OK, N.lib.cetra_last_error(ctx.handle)
        assert _static_status(N, ctx) == 0
        torch.cuda.synchronize()
        r = {k: v.cpu().numpy() for k, v in ref.items()}
        g = {k: v.cpu().numpy() for k, v in got.items()}
        np.testing.assert_array_equal(g["i"], r["i"])
        np.testing.assert_array_equal(g["j"], r["j"])
        null = np.isnan(r["dlogl"])
        np.testing.assert_array_equal(np.isnan(g["dlogl"]), null)
        if m is None:
            assert not null.any()
        else:
            assert null[:9].all() and not null[9:].all()
        for k in ("dlogl", "t0", "duration", "depth", "depth_var"):
            np.testing.assert_allclose(g[k][~null], r[k][~null], rtol=1e-6, atol=0)

    # a bounded wait that gave up is reported through the static status word ...
    rc = N.lib.cetra_selftest_static_timeout(ctx.handle)
    assert rc == N.CETRA_OK, N.lib.cetra_last_error(ctx.handle)
    assert _static_status(N, ctx) == N.CETRA_ETIMEOUT
    # ... and the next call clears it and searches normally
    periods = calls[1][0]
    d_P = torch.as_tensor(periods, device=dev)
    got = _outputs(torch, periods.size, dev)
    rc = N.lib.cetra_periodic_device_static(
        ctx.handle, plan.handle, _ptr(ws), grid_bytes, _ptr(d_P), periods.size, None,
        _ptr(got["dlogl"]), _ptr(got["t0"]), _ptr(got["duration"]), _ptr(got["depth"]),
        _ptr(got["depth_var"]), _ptr(got["i"]), _ptr(got["j"]))
    assert rc == N.CETRA_OK, N.lib.cetra_last_error(ctx.handle)
    assert _static_status(N, ctx) == 0
    assert not np.isnan(got["dlogl"].cpu().numpy()).any()

    # sizes beyond the static array are refused before any device work
    big = N.CETRA_STATIC_MAX_PERIODS + 1
    rc = N.lib.cetra_periodic_device_static(ctx.handle, plan.handle, _ptr(ws), grid_bytes,
                                            _ptr(ws), big, None, None, None, None, None, None,
                                            None, None)
    assert rc == N.CETRA_ECAPACITY
    assert b"static scratch limit" in N.lib.cetra_last_error(ctx.handle)
