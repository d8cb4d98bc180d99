"""The FP32 FMA-rate probe that gives the CUDA-core roofline its measured denominator: a positive
rate no larger than twice the nominal figure of the device (148 SMs x 128 lanes x 2 flop at
2.032 GHz = 77 TFLOP/s on a B300), and a timed launch of non-zero length."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_rate_probe():
    import paper_2111_14999_b300 as pg
    with pg.PhoebeGPU(0) as ctx:
        tflops, ms = ctx.fp32_rate()
    print(f"FP32 FMA rate {tflops:.1f} TFLOP/s ({ms:.3f} ms launch)")
    assert ms > 0.0
    assert 1.0 < tflops < 2 * 77.0
