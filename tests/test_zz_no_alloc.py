"""fwbf_decode_noalloc, the entry point for callers that cannot allocate
device memory (its frame counter lives in a fixed array of the library
instead of a per-call allocation), gives the same decisions and pass counts
as fwbf_decode, call after call.  This file is collected last so that a run
stopping at its first failure has already run every other test."""
import numpy as np
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


def test_noalloc_decode_matches_decode_on_consecutive_calls(fwbf):
    from paper_1206_3362_gb300.inputs import Encoder, bpsk_awgn, make_code, random_codewords

    h = make_code("eg1023")
    enc = Encoder(h)
    _, c = random_codewords(enc, 3000, seed=77)
    y = torch.from_numpy(bpsk_awgn(c, 3.75, enc.rate, seed=77)).cuda()
    with fwbf.Code.from_parity_check(h, 31) as code:
        q = fwbf.quantize(y)
        ref_bits, ref_iters = code.decode(q, 100, 1.5)
        torch.cuda.synchronize()
        # integer path: the tolerance is exact equality
        for call, frames in enumerate((3000, 2999)):
            bits = torch.full((frames, code.words), -7, dtype=torch.int32, device="cuda")
            iters = torch.full((frames,), -7, dtype=torch.int32, device="cuda")
            fwbf.fwbf_decode_noalloc(code.handle, q[:frames], 100, 1.5, bits, iters)
            torch.cuda.synchronize()
            assert fwbf.fwbf_last_status() == 0
            assert torch.equal(iters, ref_iters[:frames]), f"call {call}: pass counts differ"
            assert torch.equal(bits, ref_bits[:frames]), f"call {call}: decisions differ"
