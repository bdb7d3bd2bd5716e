"""Peak-rate probes of the running GPU (the roofline denominators).

Each probe keeps one pipe busy; the measured rates must be positive, finite
and ordered as the architecture fixes them: FP32 FMA above FP64 FMA, the
tensor-core rates above the FMA rates of their input widths, BF16 tensor
above TF32 tensor; and the FP64 FMA rate cannot exceed the pipe's
unit-count bound 152 SMs x 2 DFMA/clk x 2 flop x the maximum SM clock.
"""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_peaks_are_ordered_and_bounded(record_property):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_27863_gb300 import build
    build.build()
    from paper_2608_27863_gb300 import hdg as H
    t, ms = H.hdg_measure_peaks()
    record_property("tflops", t)
    assert all(math.isfinite(v) and v > 0 for v in t.values()), t
    assert t["fp32_fma"] > 4 * t["fp64_fma"]
    assert t["tf32_tcgen05"] > t["fp32_fma"] and t["bf16_tcgen05"] > t["tf32_tcgen05"]
    assert t["fp64_fma"] <= 152 * 2 * 2 * 2.07e9 / 1e12 * 1.02
