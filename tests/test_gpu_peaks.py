"""The roofline microbenchmarks (vr_measure_peaks) return plausible, finite ceilings."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    import torch
    from paper_1609_01317_gb300 import build, vr

    build.build()
    pk = vr.vr_measure_peaks(0, 3)
    props = torch.cuda.get_device_properties(0)
    for k, v in pk.items():
        assert math.isfinite(v) and v > 0.0, (k, v)
    # 128 FP32 lanes per SM at no more than 3 GHz bound the FMA rate from above
    assert pk["fma_tflops"] < props.multi_processor_count * 128 * 2 * 3.0e9 / 1e12
    assert pk["fma_tflops"] > 0.2 * props.multi_processor_count * 128 * 2 * 1.0e9 / 1e12
    # a sample's gather moves 128 bytes through L1: far below 100 TB/s of gathered bytes
    for k in ("gather_coherent_gsps", "gather_random_gsps"):
        assert pk[k] * 128 < 100e3
    # the 8 voxels of a cell in 16-bit storage are 16 bytes per sample
    for k in ("gather_u16_random_gsps", "gather_u16_coherent_gsps"):
        assert pk[k] * 16 < 100e3
