"""The FP32 FMA throughput probe (sfg_fp32_peak) that the evaluation
kernels' roofline is taken against: a plausible GB300 figure (the derived
peak is 152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s) and
repeatable to 10%."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible_and_repeatable():
    import torch
    import paper_2010_11254_gb300 as sfg
    props = torch.cuda.get_device_properties(0)
    derived = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    a = sfg.fp32_peak()
    b = sfg.fp32_peak()
    for r in (a, b):
        assert r["ms"] > 0.0
        assert 0.3 * derived < r["tflops"] < 1.05 * derived, (r, derived)
    assert abs(a["tflops"] - b["tflops"]) <= 0.1 * max(a["tflops"], b["tflops"])
