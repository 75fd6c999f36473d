"""Python face of the CETRA library: thin wrappers over the C ABI (include/cetra.h).

Host-buffer calls take numpy arrays; device calls take torch CUDA tensors
(PyTorch supplies device memory and streams only). Every stage of the search
runs in the library's CUDA kernels; nothing here computes any of it.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as N
from ._native import check


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())  # torch tensor


def _dptr(t, dtype=None, numel=0, name="tensor", optional=False):
    """Pointer of a device tensor after checking it: a contiguous CUDA torch tensor of the
    given dtype (a torch dtype name) with at least `numel` elements. A host array or a short
    buffer would reach a kernel as a bad address, so it is refused here."""
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name}: a CUDA tensor is required")
    if not hasattr(t, "is_cuda") or not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA torch tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if dtype is not None and str(t.dtype) != "torch." + dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected torch.{dtype}")
    if t.numel() < numel:
        raise ValueError(f"{name}: {t.numel()} elements, at least {numel} needed")
    return ctypes.c_void_p(t.data_ptr())


def _wsb(ws):
    """(pointer, bytes) of a device workspace tensor."""
    return _dptr(ws, name="workspace"), ws.numel() * ws.element_size()


def make_params(cadence=0.0, t0_step=0.0, template_samples=1024, flux_is_offset=False,
                precision="fp32") -> N.cetra_params:
    p = N.cetra_params()
    N.lib.cetra_params_default(ctypes.byref(p))
    p.cadence = float(cadence or 0.0)
    p.t0_step = float(t0_step or 0.0)
    p.template_samples = int(template_samples)
    p.flux_is_offset = int(bool(flux_is_offset))
    p.precision = {"fp32": N.CETRA_FP32, "kahan": N.CETRA_FP32_KAHAN}[precision]
    return p


class Context:
    """A library context on one CUDA device, launching on one stream."""

    def __init__(self, device: int = 0, stream=None):
        self.handle = ctypes.c_void_p()
        st = _stream_handle(stream)
        check(N.lib.cetra_create(ctypes.byref(self.handle), int(device), st), None, "create")
        self.device = device

    def set_stream(self, stream):
        check(N.lib.cetra_set_stream(self.handle, _stream_handle(stream)), self.handle)

    @property
    def launches(self) -> int:
        return int(N.lib.cetra_kernel_launches(self.handle))

    def profile(self, enable: bool = True):
        check(N.lib.cetra_profile_enable(self.handle, int(bool(enable))), self.handle)

    def profile_read(self, kernel: str):
        """(launches, total device ms) of one kernel since the last read."""
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0.0)
        check(N.lib.cetra_profile_read(self.handle, kernel.encode(), ctypes.byref(n),
                                       ctypes.byref(ms)), self.handle, "profile_read")
        return int(n.value), float(ms.value)

    def close(self):
        if self.handle:
            N.lib.cetra_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _info_dict(info: N.cetra_plan_info) -> dict:
    return {f: getattr(info, f) for f, _ in N.cetra_plan_info._fields_}


class Plan:
    """Geometry and window tables of a search (cetra_plan_create)."""

    def __init__(self, ctx: Context, time, flux, flux_err, durations, tmpl, **params):
        self.ctx = ctx
        t = _np(time, np.float64)
        f = _np(flux, np.float32)
        e = _np(flux_err, np.float32)
        d = _np(durations, np.float64)
        tm = _np(tmpl, np.float32)
        self.durations = d
        self.params = make_params(**params)
        self.handle = ctypes.c_void_p()
        check(N.lib.cetra_plan_create(ctx.handle, ctypes.byref(self.params), _ptr(t), _ptr(f),
                                      _ptr(e), t.size, _ptr(d), d.size, _ptr(tm), tm.size,
                                      ctypes.byref(self.handle)), ctx.handle, "plan_create")
        info = N.cetra_plan_info()
        check(N.lib.cetra_plan_get_info(self.handle, ctypes.byref(info)), ctx.handle)
        self.info = _info_dict(info)

    def workspace_bytes(self, n_periods: int = 0) -> int:
        return int(N.lib.cetra_workspace_bytes(self.handle, int(n_periods)))

    def t0_grid(self) -> np.ndarray:
        """Mid-times t_i (absolute days) of the t0 grid."""
        i = np.arange(self.info["n_t0"], dtype=np.int64)
        ticks = i * self.info["p"] - self.info["n_pad"] * self.info["q"]
        return self.info["t_ref"] + ticks * self.info["cadence"] / self.info["q"]

    def close(self):
        if self.handle:
            N.lib.cetra_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- device path

def cetra_resample_device(ctx: Context, plan: Plan, d_time, d_flux, d_flux_err, workspace):
    n = int(d_time.numel())
    ws, nb = _wsb(workspace)
    check(N.lib.cetra_resample_device(ctx.handle, plan.handle, _dptr(d_time, "float64", n, "time"),
                                      _dptr(d_flux, "float32", n, "flux"),
                                      _dptr(d_flux_err, "float32", n, "flux_err"), n, ws, nb),
          ctx.handle, "resample_device")


def cetra_linear_device(ctx: Context, plan: Plan, workspace, d_depth=None, d_depth_var=None,
                        d_dlogl=None):
    cells = plan.info["n_dur"] * plan.info["n_t0"]
    ws, nb = _wsb(workspace)
    check(N.lib.cetra_linear_device(ctx.handle, plan.handle, ws, nb,
                                    _dptr(d_depth, "float32", cells, "depth", True),
                                    _dptr(d_depth_var, "float32", cells, "depth_var", True),
                                    _dptr(d_dlogl, "float32", cells, "dlogl", True)),
          ctx.handle, "linear_device")


def cetra_periodic_device(ctx: Context, plan: Plan, workspace, d_periods, d_mask=None,
                          out: dict | None = None):
    out = out or {}
    K = int(d_periods.numel())
    ws, nb = _wsb(workspace)
    o = {k: _dptr(out.get(k), dt, K, k, True) for k, dt in
         (("dlogl", "float64"), ("t0", "float64"), ("duration", "float64"),
          ("depth", "float64"), ("depth_var", "float64"), ("i", "int64"), ("j", "int32"))}
    check(N.lib.cetra_periodic_device(ctx.handle, plan.handle, ws, nb,
                                      _dptr(d_periods, "float64", K, "periods"), K,
                                      _dptr(d_mask, "uint8", K * plan.info["n_dur"], "mask", True),
                                      o["dlogl"], o["t0"], o["duration"], o["depth"],
                                      o["depth_var"], o["i"], o["j"]),
          ctx.handle, "periodic_device")


def cetra_logl0_device(ctx: Context, plan: Plan, workspace, d_out):
    ws, nb = _wsb(workspace)
    check(N.lib.cetra_logl0_device(ctx.handle, plan.handle, ws, nb,
                                   _dptr(d_out, "float64", 1, "logl0")),
          ctx.handle, "logl0_device")


class DeviceSearch:
    """Device buffers (torch) for one plan and one period grid, and the three
    stages run on them: resample -> linear -> periodic."""

    def __init__(self, ctx: Context, plan: Plan, periods, mask=None, linear_outputs=True):
        import torch
        dev = torch.device("cuda", ctx.device)
        self.ctx, self.plan = ctx, plan
        K = int(np.size(periods))
        self.K = K
        self.workspace = torch.empty(plan.workspace_bytes(K), dtype=torch.uint8, device=dev)
        self.periods = torch.as_tensor(_np(periods, np.float64), device=dev)
        self.mask = None if mask is None else torch.as_tensor(_np(mask, np.uint8), device=dev)
        J, I = plan.info["n_dur"], plan.info["n_t0"]
        if linear_outputs:
            self.depth = torch.empty((J, I), dtype=torch.float32, device=dev)
            self.depth_var = torch.empty_like(self.depth)
            self.dlogl = torch.empty_like(self.depth)
        else:
            self.depth = self.depth_var = self.dlogl = None
        self.out = {k: torch.empty(K, dtype=torch.float64, device=dev)
                    for k in ("dlogl", "t0", "duration", "depth", "depth_var")}
        self.out["i"] = torch.empty(K, dtype=torch.int64, device=dev)
        self.out["j"] = torch.empty(K, dtype=torch.int32, device=dev)
        self.logl0 = torch.empty(1, dtype=torch.float64, device=dev)

    def run(self, d_time, d_flux, d_flux_err, periodic=True, logl0=False):
        cetra_resample_device(self.ctx, self.plan, d_time, d_flux, d_flux_err, self.workspace)
        cetra_linear_device(self.ctx, self.plan, self.workspace, self.depth, self.depth_var,
                            self.dlogl)
        if logl0:
            cetra_logl0_device(self.ctx, self.plan, self.workspace, self.logl0)
        if periodic and self.K:
            cetra_periodic_device(self.ctx, self.plan, self.workspace, self.periods, self.mask,
                                  self.out)
        return self


def cetra_mask_transits_device(ctx: Context, plan: Plan, d_workspace, period, t0, half_width,
                               d_n_masked=None):
    """Null the resampled cells within half_width days of t0 + n period (then rerun
    cetra_linear_device)."""
    ws, nb = _wsb(d_workspace)
    check(N.lib.cetra_mask_transits_device(ctx.handle, plan.handle, ws, nb, float(period),
                                           float(t0), float(half_width),
                                           _dptr(d_n_masked, "int64", 1, "n_masked", True)),
          ctx.handle, "mask_transits_device")


def cetra_monotransits_device(ctx: Context, plan: Plan, d_workspace, max_events, d_events, d_n):
    """Single-transit events into d_events (a device byte tensor of max_events records)
    and d_n (device int32)."""
    ws, nb = _wsb(d_workspace)
    rec = ctypes.sizeof(N.cetra_event)
    if d_events is None or d_events.numel() * d_events.element_size() < int(max_events) * rec:
        raise ValueError(f"events: needs {int(max_events) * rec} bytes of device memory")
    check(N.lib.cetra_monotransits_device(ctx.handle, plan.handle, ws, nb, int(max_events),
                                          _dptr(d_events, None, 0, "events"),
                                          _dptr(d_n, "int32", 1, "n_events")),
          ctx.handle, "monotransits_device")


def cetra_selftest_wait_timeout(ctx: Context):
    """Run the bounded-wait self-test: (timed_out, seconds)."""
    flag, secs = ctypes.c_int(0), ctypes.c_double(0.0)
    check(N.lib.cetra_selftest_wait_timeout(ctx.handle, ctypes.byref(flag), ctypes.byref(secs)),
          ctx.handle, "selftest_wait_timeout")
    return flag.value, secs.value


def cetra_measure_peaks(ctx: Context):
    """Measured ceilings of the two stages' bounds: (FP32 FMA TFLOP/s, shared-load GB/s)."""
    fma, smem = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(N.lib.cetra_measure_peaks(ctx.handle, ctypes.byref(fma), ctypes.byref(smem)),
          ctx.handle, "measure_peaks")
    return fma.value, smem.value


def events_dict(events):
    """Records of cetra_event -> dict of numpy arrays."""
    return {f: np.array([getattr(e, f) for e in events])
            for f, _ in N.cetra_event._fields_ if f != "pad_"}


# ----------------------------------------------------------------------------- host-buffer path

class LinearGrid:
    """Device-resident result of cetra_linear_search (owns its device memory)."""

    def __init__(self, ctx: Context, handle):
        self.ctx, self.handle = ctx, handle
        info = N.cetra_plan_info()
        check(N.lib.cetra_grid_get_info(handle, ctypes.byref(info)), ctx.handle)
        self.info = _info_dict(info)

    def close(self):
        if self.handle:
            N.lib.cetra_grid_free(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cetra_linear_search(ctx: Context, time, flux, flux_err, durations, tmpl, *, outputs=True,
                        keep_grid=True, **params):
    """Linear search (Sec. 2.2) on host arrays. Returns (grid, depth, depth_var, dlogl)."""
    t = _np(time, np.float64)
    f = _np(flux, np.float32)
    e = _np(flux_err, np.float32)
    d = _np(durations, np.float64)
    tm = _np(tmpl, np.float32)
    prm = make_params(**params)
    n_t0 = ctypes.c_int64(0)
    grid = ctypes.c_void_p()
    depth = var = lr = None
    if outputs:
        info = N.cetra_plan_info()
        check(N.lib.cetra_plan_geometry(ctx.handle, ctypes.byref(prm), _ptr(t), _ptr(f), _ptr(e),
                                        t.size, _ptr(d), d.size, ctypes.byref(info)),
              ctx.handle, "plan_geometry")
        I = info.n_t0
        n_t0.value = I
        depth = np.empty((d.size, I), np.float32)
        var = np.empty((d.size, I), np.float32)
        lr = np.empty((d.size, I), np.float32)
    check(N.lib.cetra_linear_search(ctx.handle, ctypes.byref(prm), _ptr(t), _ptr(f), _ptr(e),
                                    t.size, _ptr(d), d.size, _ptr(tm), tm.size,
                                    ctypes.byref(grid) if keep_grid else None, _ptr(depth),
                                    _ptr(var), _ptr(lr), ctypes.byref(n_t0)),
          ctx.handle, "linear_search")
    return (LinearGrid(ctx, grid) if keep_grid else None), depth, var, lr


def cetra_mask_transits(ctx: Context, grid: LinearGrid, period, t0, half_width) -> int:
    """Mask a grid around t0 + n period (half_width days) and rerun its linear stage;
    returns the number of nulled cells that held data."""
    n = ctypes.c_int64(0)
    check(N.lib.cetra_mask_transits(ctx.handle, grid.handle, float(period), float(t0),
                                    float(half_width), ctypes.byref(n)), ctx.handle,
          "mask_transits")
    return n.value


def cetra_monotransit_search(ctx: Context, grid: LinearGrid, max_events=10) -> dict:
    """Up to max_events single-transit events of a grid, strongest first."""
    ev = (N.cetra_event * int(max_events))()
    n = ctypes.c_int(0)
    check(N.lib.cetra_monotransit_search(ctx.handle, grid.handle, int(max_events), ev,
                                         ctypes.byref(n)), ctx.handle, "monotransit_search")
    return events_dict(list(ev)[:n.value])


def cetra_search_iterative(ctx: Context, grid: LinearGrid, periods, n_iter=3, width=2.0,
                           mask=None) -> dict:
    """n_iter rounds of the periodic search, masking each round's best signal (Sec. 4.2)."""
    P = _np(periods, np.float64)
    m = None if mask is None else _np(mask, np.uint8)
    out = (N.cetra_best * int(n_iter))()
    n = ctypes.c_int(0)
    check(N.lib.cetra_search_iterative(ctx.handle, grid.handle, _ptr(P), P.size, _ptr(m),
                                       int(n_iter), float(width), out, ctypes.byref(n)),
          ctx.handle, "search_iterative")
    return _best_dict(list(out)[:n.value])


def cetra_periodic_search(ctx: Context, grid: LinearGrid, periods, mask=None) -> dict:
    """Periodic search (Sec. 2.3) on a grid from cetra_linear_search; host outputs."""
    P = _np(periods, np.float64)
    m = None if mask is None else _np(mask, np.uint8)
    K = P.size
    out = {k: np.empty(K, np.float64) for k in ("dlogl", "t0", "duration", "depth", "depth_var")}
    best = ctypes.c_int64(-1)
    check(N.lib.cetra_periodic_search(ctx.handle, grid.handle, _ptr(P), K, _ptr(m),
                                      _ptr(out["dlogl"]), _ptr(out["t0"]), _ptr(out["duration"]),
                                      _ptr(out["depth"]), _ptr(out["depth_var"]),
                                      ctypes.byref(best)), ctx.handle, "periodic_search")
    out["best_k"] = best.value
    return out


# ----------------------------------------------------------------------------- batched form

BEST_FIELDS = [f for f, _ in N.cetra_best._fields_]


def batch_period_grid(period_min, ratio, n_periods):
    """Periods 0 .. n_periods-1 of a batch curve: period_min * ratio^k with ratio^k by
    LSB-first square-and-multiply in FP64 (the definition cetra_batch_create uses)."""
    k = np.arange(int(n_periods), dtype=np.int64)
    x = np.ones(k.size)
    b = np.full(k.size, float(ratio))
    m = k.copy()
    while np.any(m):
        x = np.where(m & 1, x * b, x)
        b = b * b
        m >>= 1
    return float(period_min) * x


def _best_dict(arr):
    return {f: np.array([getattr(b, f) for b in arr]) for f in BEST_FIELDS}


def _pack(curves):
    """CSR packing of a list of (time, flux, flux_err) arrays."""
    lens = [len(c[0]) for c in curves]
    off = np.zeros(len(curves) + 1, np.int64)
    off[1:] = np.cumsum(lens)
    t = np.ascontiguousarray(np.concatenate([np.asarray(c[0], np.float64) for c in curves]))
    f = np.ascontiguousarray(np.concatenate([np.asarray(c[1], np.float32) for c in curves]))
    e = np.ascontiguousarray(np.concatenate([np.asarray(c[2], np.float32) for c in curves]))
    return off, t, f, e


class Batch:
    """cetra_batch_create / run / destroy over a list of (time, flux, flux_err) curves."""

    def __init__(self, ctx: Context, curves, durations, tmpl, period_min, period_max=None,
                 period_ratio=None, autotune=False, csr=None, **params):
        """curves: a list of (time, flux, flux_err); or csr = (offsets [n + 1], time, flux,
        flux_err) already packed back to back (then curves is ignored)."""
        self.ctx = ctx
        if csr is not None:
            off = _np(csr[0], np.int64)
            t, f, e = _np(csr[1], np.float64), _np(csr[2], np.float32), _np(csr[3], np.float32)
        else:
            off, t, f, e = _pack(curves)
        n = off.size - 1
        d = _np(durations, np.float64)
        tm = _np(tmpl, np.float32)
        pmin = _np(np.broadcast_to(period_min, (n,)), np.float64)
        pmax = None if period_max is None else _np(np.broadcast_to(period_max, (n,)), np.float64)
        rat = None if period_ratio is None else _np(np.broadcast_to(period_ratio, (n,)), np.float64)
        self.params = make_params(**params)
        self.handle = ctypes.c_void_p()
        self._keep = (off, t, f, e, d, tm, pmin, pmax, rat)
        check(N.lib.cetra_batch_create(ctx.handle, ctypes.byref(self.params), n, _ptr(off),
                                       _ptr(t), _ptr(f), _ptr(e), _ptr(d), d.size, _ptr(tm),
                                       tm.size, _ptr(pmin), _ptr(pmax), _ptr(rat),
                                       int(bool(autotune)), ctypes.byref(self.handle)),
              ctx.handle, "batch_create")
        self.n = n

    @property
    def info(self) -> dict:
        info = N.cetra_batch_info()
        check(N.lib.cetra_batch_get_info(self.handle, ctypes.byref(info)), self.ctx.handle)
        return {f: getattr(info, f) for f, _ in N.cetra_batch_info._fields_}

    def run(self, results=True):
        best = (N.cetra_best * self.n)() if results else None
        check(N.lib.cetra_batch_run(self.ctx.handle, self.handle, best), self.ctx.handle,
              "batch_run")
        return _best_dict(best) if results else None

    def features(self, n_bins=4096, out=None):
        """Max-pooled linear LR [n_curves][n_dur][n_bins] (torch CUDA tensor; written into
        `out` when given, a contiguous tensor of that shape)."""
        import torch
        J = self.info["n_dur"]
        if out is None:
            out = torch.empty((self.n, J, n_bins), dtype=torch.float32,
                              device=torch.device("cuda", self.ctx.device))
        elif tuple(out.shape) != (self.n, J, n_bins) or not out.is_contiguous():
            raise ValueError("out must be a contiguous [n_curves][n_dur][n_bins] tensor")
        check(N.lib.cetra_batch_features(self.ctx.handle, self.handle, int(n_bins),
                                         _dptr(out, "float32", self.n * J * n_bins, "out")),
              self.ctx.handle, "batch_features")
        return out

    def curve(self, c):
        """(t_ref, period_min, ratio, n_periods, n_t0, first_item) of curve c."""
        t_ref, pmin, rat = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        K, I, first = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        check(N.lib.cetra_batch_curve(self.handle, int(c), ctypes.byref(t_ref), ctypes.byref(pmin),
                                      ctypes.byref(rat), ctypes.byref(K), ctypes.byref(I),
                                      ctypes.byref(first)), self.ctx.handle, "batch_curve")
        return t_ref.value, pmin.value, rat.value, K.value, I.value, first.value

    def run_items(self, items, linear=True):
        """Fold only the listed (curve, 8-period group) items; per-curve best."""
        it = _np(items, np.int64)
        best = (N.cetra_best * self.n)()
        check(N.lib.cetra_batch_run_items(self.ctx.handle, self.handle, _ptr(it), it.size,
                                          int(bool(linear)), best), self.ctx.handle,
              "batch_run_items")
        return _best_dict(best)

    def run_proposed(self, d_scores, p_lo, p_hi, top_frac, linear=False, items=False):
        """Fold each curve's best-scored period intervals (selection on the device).
        Returns (best dict, n_items, n_periods[, items])."""
        if tuple(d_scores.shape[:1]) != (self.n,) or not d_scores.is_contiguous():
            raise ValueError("d_scores must be a contiguous [n_curves][n_intervals] tensor")
        best = (N.cetra_best * self.n)()
        n_it, n_per = ctypes.c_int64(), ctypes.c_int64()
        buf = np.empty(max(1, self.info["n_fold_items"]), np.int64) if items else None
        n_int = int(d_scores.shape[1]) if d_scores.dim() == 2 else 0
        check(N.lib.cetra_batch_run_proposed(self.ctx.handle, self.handle,
                                             _dptr(d_scores, "float32", self.n * n_int, "scores"),
                                             int(d_scores.shape[1]), float(p_lo), float(p_hi),
                                             float(top_frac), int(bool(linear)), best,
                                             ctypes.byref(n_it), ctypes.byref(n_per), _ptr(buf)),
              self.ctx.handle, "batch_run_proposed")
        out = (_best_dict(best), n_it.value, n_per.value)
        return out + (np.sort(buf[:n_it.value]),) if items else out

    def search_proposed(self, cnn, n_intervals=512, p_lo=0.5, p_hi=0.0, top_frac=0.05):
        """The whole learned-proposal search in one library call (cetra_batch_search_proposed).
        Returns (best dict, n_items, n_periods)."""
        best = (N.cetra_best * self.n)()
        n_it, n_per = ctypes.c_int64(), ctypes.c_int64()
        check(N.lib.cetra_batch_search_proposed(self.ctx.handle, self.handle, cnn.handle,
                                                int(n_intervals), float(p_lo), float(p_hi),
                                                float(top_frac), best, ctypes.byref(n_it),
                                                ctypes.byref(n_per)),
              self.ctx.handle, "batch_search_proposed")
        return _best_dict(best), n_it.value, n_per.value

    def close(self):
        if self.handle:
            N.lib.cetra_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cetra_search_batch(ctx: Context, curves, durations, tmpl, period_min, period_max=None,
                       period_ratio=None, **params) -> dict:
    """One-shot batched search (host buffers in, per-curve best model out)."""
    off, t, f, e = _pack(curves)
    n = len(curves)
    d = _np(durations, np.float64)
    tm = _np(tmpl, np.float32)
    pmin = _np(np.broadcast_to(period_min, (n,)), np.float64)
    pmax = None if period_max is None else _np(np.broadcast_to(period_max, (n,)), np.float64)
    rat = None if period_ratio is None else _np(np.broadcast_to(period_ratio, (n,)), np.float64)
    prm = make_params(**params)
    best = (N.cetra_best * n)()
    check(N.lib.cetra_search_batch(ctx.handle, ctypes.byref(prm), n, _ptr(off), _ptr(t), _ptr(f),
                                   _ptr(e), _ptr(d), d.size, _ptr(tm), tm.size, _ptr(pmin),
                                   _ptr(pmax), _ptr(rat), best), ctx.handle, "search_batch")
    return _best_dict(best)


# ----------------------------------------------------------------------------- learned proposal

class CNN:
    """The period-interval proposal network (cetra_cnn_*)."""

    def __init__(self, ctx: Context, in_channels, n_bins=4096, max_batch=64, seed=1):
        self.ctx = ctx
        self.handle = ctypes.c_void_p()
        check(N.lib.cetra_cnn_create(ctx.handle, int(in_channels), int(n_bins), int(max_batch),
                                     int(seed), ctypes.byref(self.handle)), ctx.handle,
              "cnn_create")
        self.n_params = int(N.lib.cetra_cnn_param_count(self.handle))
        self.n_bins = n_bins
        self.in_channels = in_channels
        self.max_batch = max_batch

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        check(N.lib.cetra_cnn_get_params(self.ctx.handle, self.handle, _ptr(out)), self.ctx.handle)
        return out

    def set_params(self, params):
        p = _np(params, np.float32)
        assert p.size == self.n_params
        check(N.lib.cetra_cnn_set_params(self.ctx.handle, self.handle, _ptr(p)), self.ctx.handle)

    def _features(self, d_features):
        if tuple(d_features.shape[1:]) != (self.in_channels, self.n_bins):
            raise ValueError(f"features: shape {tuple(d_features.shape)}, expected "
                             f"[B][{self.in_channels}][{self.n_bins}]")
        B = int(d_features.shape[0])
        return B, _dptr(d_features, "float32", B * self.in_channels * self.n_bins, "features")

    def forward(self, d_features, d_prob):
        B, f = self._features(d_features)
        check(N.lib.cetra_cnn_forward(self.ctx.handle, self.handle, f, B,
                                      _dptr(d_prob, "float32", B * self.n_bins, "prob")),
              self.ctx.handle, "cnn_forward")

    def backward(self, d_features, d_labels, pos_weight=20.0, grads=False):
        loss = ctypes.c_double(0.0)
        g = np.empty(self.n_params, np.float32) if grads else None
        B, f = self._features(d_features)
        check(N.lib.cetra_cnn_backward(self.ctx.handle, self.handle, f,
                                       _dptr(d_labels, "float32", B * self.n_bins, "labels"), B,
                                       float(pos_weight), ctypes.byref(loss), _ptr(g)),
              self.ctx.handle, "cnn_backward")
        return (loss.value, g) if grads else loss.value

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        check(N.lib.cetra_cnn_adam(self.ctx.handle, self.handle, float(lr), float(beta1),
                                   float(beta2), float(eps)), self.ctx.handle, "cnn_adam")

    def close(self):
        if self.handle:
            N.lib.cetra_cnn_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cetra_cnn_map(ctx: Context, d_prob, d_features, d_map):
    """d_map = d_prob * (max over durations of d_features, clipped at 0) (device tensors)."""
    B, J, T = (int(x) for x in d_features.shape)
    check(N.lib.cetra_cnn_map(ctx.handle, _dptr(d_prob, "float32", B * T, "prob"),
                              _dptr(d_features, "float32", B * J * T, "features"), B, J, T,
                              _dptr(d_map, "float32", B * T, "map")), ctx.handle, "cnn_map")


def cetra_cnn_comb(ctx: Context, d_map, d_bin_days, p_lo, p_hi, n_intervals, d_scores,
                   d_n_valid=None):
    B, T = (int(x) for x in d_map.shape)
    check(N.lib.cetra_cnn_comb(ctx.handle, _dptr(d_map, "float32", B * T, "map"), B, T,
                               _dptr(d_bin_days, "float64", B, "bin_days"),
                               _dptr(d_n_valid, "int32", B, "n_valid", True), float(p_lo),
                               float(p_hi), int(n_intervals),
                               _dptr(d_scores, "float32", B * int(n_intervals), "scores")),
          ctx.handle, "cnn_comb")
