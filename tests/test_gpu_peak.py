"""The integer issue-rate microbenchmark (the decoder roofline's measured
denominator) reports rates the GPU's unit counts allow."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fwbf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1206_3362_gb300 import fwbf as mod

    return mod


def test_int_issue_rate_within_unit_counts(fwbf):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    logic = fwbf.fwbf_peak_int_issue(0, 50.0)
    mixed = fwbf.fwbf_peak_int_issue(1, 50.0)
    # at most 128 lanes per SM per clock at 2.2 GHz; at least a quarter of that at 1 GHz
    ceiling = sms * 128 * 2.2e9
    assert 0.0 < logic <= mixed <= ceiling
    assert mixed >= sms * 32 * 1.0e9
