"""The roofline microbenchmarks: packed FP32 FMA chains and 8-byte shared-memory loads (the
linear search's and the fold's bounds) measure rates no higher than the SM's nominal ones."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_within_nominal():
    import torch
    from paper_2503_20875_gb300 import Context, cetra_measure_peaks
    ctx = Context(0)
    fma, smem = cetra_measure_peaks(ctx)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ghz = 2.2  # above any GB300 SM clock
    fma_nominal = sms * 128 * 2 * ghz * 1e-3         # TFLOP/s
    smem_nominal = sms * 128 * ghz                   # GB/s at 128 B/clk/SM
    msg = f"FP32 FMA {fma:.1f} TFLOP/s, shared loads {smem:.0f} GB/s"
    print(msg)
    assert math.isfinite(fma) and 0.3 * fma_nominal < fma <= fma_nominal, msg
    # above the nominal rate would mean loads were lifted out of the timed loop
    assert math.isfinite(smem) and 0.1 * smem_nominal < smem <= smem_nominal, msg
