"""Failure detection without a GPU fault: every barrier wait of the fold is bounded; a kernel
that waits on a barrier no copy will complete must give up after about a second, report it,
and leave the context usable for the next search."""
import numpy as np
import pytest

import oracle
from synth.lightcurves import custom, HOUR
from tests._parity import gpu_search

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_survives():
    from paper_2503_20875_gb300 import Context
    from paper_2503_20875_gb300.api import cetra_selftest_wait_timeout
    ctx = Context(0)
    timed_out, seconds = cetra_selftest_wait_timeout(ctx)
    assert timed_out == 1
    assert 0.1 < seconds < 30.0
    # the same process then searches a curve and matches the oracle
    w = custom(seed=3, n_points=1500, durations_h=(1.0, 2.0),
               planets=[dict(P=1.1, t0=0.3, D=2.0 * HOUR, depth=3e-3)])
    periods = np.exp(np.linspace(np.log(0.5), np.log(1.8), 60))
    got = gpu_search(w.time, w.flux, w.flux_err, w.durations, w.template, periods,
                     cadence=w.cadence, t0_step=w.t0_step)
    ref = oracle.search(w.time, w.flux, w.flux_err, w.durations, w.template, periods,
                        cadence=w.cadence, t0_step=w.t0_step)
    k = int(np.nanargmax(ref["periodic"]["dlogl"]))
    assert int(np.nanargmax(got["periodic"]["dlogl"])) == k
    assert got["periodic"]["dlogl"][k] == pytest.approx(ref["periodic"]["dlogl"][k], rel=1e-5)
