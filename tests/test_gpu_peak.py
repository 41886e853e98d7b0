"""Diagnostics: the integer issue-rate microbenchmark (the decoder roofline's
measured denominator) reports rates the GPU's unit counts allow; the bounded
wait of the table staging gives up with FWBF_ETIMEOUT (a barrier nothing
completes, no GPU fault) and leaves the context usable."""
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


def test_bounded_wait_reports_timeout(fwbf):
    import time

    import numpy as np

    import oracle
    from paper_1206_3362_gb300.inputs import Encoder, bpsk_awgn, make_code, random_codewords

    assert fwbf.fwbf_probe_bounded_wait(0) == fwbf.FWBF_OK
    t0 = time.time()
    assert fwbf.fwbf_probe_bounded_wait(16) == fwbf.FWBF_ETIMEOUT
    assert 0.9 < time.time() - t0 < 30.0
    # the context still decodes
    h = make_code("eg255")
    enc = Encoder(h)
    _, c = random_codewords(enc, 40, seed=3)
    q = oracle.quantize(bpsk_awgn(c, 4.0, enc.rate, seed=3))
    with fwbf.Code.from_parity_check(h, 16) as code:
        bits, iters = code.decode(torch.from_numpy(q).cuda(), 30, 1.5)
        torch.cuda.synchronize()
    bo, io = oracle.fwbf_i8(h, 16, q, 30, 1.5)
    assert np.array_equal(iters.cpu().numpy(), io)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), bo)
