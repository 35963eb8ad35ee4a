"""The peak probes report rates within the physical range of the part.

FP32: 152 SMs x 128 lanes x 2 flops x the SM clock (at most about 2.1 GHz)
bounds the f32x2 FMA rate near 81 TFLOP/s.  TF32: the dense tensor rate is
about half the BF16 rate (nominal 2.25 PFLOP/s BF16, 1.1 TF32); FP16 runs at
the BF16 rate and above the TF32 rate (measured up to 2.41 PFLOP/s, a little
above the nominal dense figure at the part's top clock; bound at 2.7).  Each rate
must come out positive and below those ceilings, and above a floor that a
mis-timed or dropped kernel would miss."""
import pytest

from paper_1606_02383_gb300 import _lib, peaks

pytestmark = pytest.mark.gpu


def test_fp32_tf32_and_fp16_rates_in_range(cuda_ok):
    fp32 = peaks.measure("fp32")
    tf32 = peaks.measure("tf32")
    fp16 = peaks.measure("fp16")
    assert 30.0 < fp32 < 90.0, fp32
    assert 300.0 < tf32 < 1300.0, tf32
    assert tf32 < fp16 < 2700.0, (tf32, fp16)


def test_probe_rejects_bad_arguments(cuda_ok):
    with pytest.raises(ValueError):
        peaks.measure("fp64")
    with pytest.raises(_lib.BemError):
        peaks.measure("fp32", iters=0)
