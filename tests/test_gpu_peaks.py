"""The device microbenchmarks behind the roofline denominators
(salt_measure_peaks): the measured FP32 FMA rate against the rate derived from
the SM count and the maximum SM clock, and sane L2 / shared-memory read
bandwidths."""
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_peaks_bracket_the_derived_fp32_peak():
    from paper_2504_08081_b300 import build
    build.build()
    from paper_2504_08081_b300.torch_api import Salt
    wl = W.config1()
    s = Salt(wl.model, wl.bands)
    pk = s.measure_peaks()
    props = torch.cuda.get_device_properties(0)
    assert pk["num_sms"] == props.multi_processor_count
    derived = pk["num_sms"] * 128 * 2 * pk["sm_clock_max_mhz"] * 1e6 / 1e12
    # at most the derived peak (small timer slack); at least 60 % of it even
    # under a power-capped clock
    assert 0.6 * derived <= pk["fp32_tflops"] <= 1.02 * derived, (pk, derived)
    assert pk["l2_read_gbs"] > 1000.0
    assert pk["smem_read_gbs"] > pk["l2_read_gbs"]
    s.close()
