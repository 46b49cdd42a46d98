"""The measured FP32 rate (s3ttv_fp32_peak), the denominator of the ALU roofline
of the eigen-solve-bound kernels: it must run, be finite, and lie between a
tenth of and just above the rate derived from the unit counts at the device's
maximum SM clock (SMs x 128 FP32 lanes x 2 flops x clock; packed FP32x2 FMAs
counted per lane, so up to twice that)."""
import math
import subprocess

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def max_sm_mhz():
    try:
        out = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=30).stdout
        return float(out.strip().splitlines()[0])
    except Exception:
        return 2070.0


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_03313_gb300 as P
    P.library()
    return P


def test_fp32_peak_is_plausible(P):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * max_sm_mhz() * 1e6 / 1e12
    scalar = P.fp32_peak(0, False)
    packed = P.fp32_peak(0, True)
    print(f"FP32 TFLOP/s: scalar {scalar:.2f}, packed {packed:.2f}, derived {derived:.2f}")
    for x in (scalar, packed):
        assert math.isfinite(x)
    assert 0.1 * derived < scalar < 1.1 * derived
    assert 0.1 * derived < packed < 2.2 * derived


def test_fp32_peak_rejects_bad_arguments(P):
    import ctypes
    t = ctypes.c_double()
    assert P.library().s3ttv_fp32_peak(0, 2, ctypes.byref(t)) == P.EINVAL
    assert P.library().s3ttv_fp32_peak(0, 0, None) == P.EINVAL
