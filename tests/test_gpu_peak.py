"""GPU: the FP32 FMA throughput measurement (dcm_fp32_peak) runs and returns a
figure between a quarter and 1.5x the unit-count peak of the device (SMs x 128
FP32 lanes x 2 flops at the highest SM clock)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1502_03234_gb300 import dcm

    tf, ms = dcm.dcm_fp32_peak(20000)
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.1e9 / 1e12
    assert 0.25 * nominal < tf < 1.5 * nominal, (tf, nominal)
    assert ms > 0
    with pytest.raises(dcm.DcmError):
        dcm.dcm_fp32_peak(0)
