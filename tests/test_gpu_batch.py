"""Batched multi-code decoding in one persistent launch: every job's results
equal fwbf_decode's (and the oracle's on sampled frames), for both decoder
variants and several CTA sizes, and a captured CUDA graph replays them."""
import numpy as np
import pytest

import oracle
from paper_1206_3362_gb300.inputs import Encoder, bpsk_awgn, make_code, random_codewords

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX = [("rand504", 32, 4), ("rand2016", 32, 2), ("eg4095", 63, 1), ("qc8192", 64, 1)]


@pytest.fixture(scope="module")
def fwbf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1206_3362_gb300 import fwbf as mod

    return mod


@pytest.fixture(scope="module")
def jobs(fwbf):
    out = []
    for i, (key, p, share) in enumerate(MIX):
        h = make_code(key)
        enc = Encoder(h)
        F = 96 * share + 7
        _, c = random_codewords(enc, F, seed=50 + i)
        q = oracle.quantize(bpsk_awgn(c, 3.75, enc.rate, seed=50 + i))
        code = fwbf.Code.from_parity_check(h, p)
        out.append(dict(key=key, h=h, p=p, q=q, qd=torch.from_numpy(q).cuda(), code=code))
    yield out
    for j in out:
        j["code"].close()


def _single(fwbf, j):
    bits, iters = j["code"].decode(j["qd"], 60, 1.5)
    torch.cuda.synchronize()
    return bits.cpu().numpy(), iters.cpu().numpy()


@pytest.mark.parametrize("warps,packed", [(16, 2), (16, 1), (8, 1), (4, 1), (16, 0), (7, 0)])
def test_batch_equals_single_code_decoding(fwbf, jobs, warps, packed):
    outs = [j["code"].outputs(j["qd"].shape[0]) for j in jobs]
    spec = [(j["code"].handle, j["qd"], 60, 1.5, b, it) for j, (b, it) in zip(jobs, outs)]
    batch = fwbf.fwbf_batch_create(spec, warps_per_cta=warps, packed=packed)
    try:
        fwbf.fwbf_decode_batch(batch)
        torch.cuda.synchronize()
        assert fwbf.fwbf_batch_status() == 0
        for j, (b, it) in zip(jobs, outs):
            sb, si = _single(fwbf, j)
            assert np.array_equal(it.cpu().numpy(), si), j["key"]
            assert np.array_equal(b.cpu().numpy(), sb), j["key"]
    finally:
        fwbf.fwbf_batch_destroy(batch)


def test_batch_matches_oracle_on_samples(fwbf, jobs):
    outs = [j["code"].outputs(j["qd"].shape[0]) for j in jobs]
    spec = [(j["code"].handle, j["qd"], 60, 1.5, b, it) for j, (b, it) in zip(jobs, outs)]
    batch = fwbf.fwbf_batch_create(spec)
    fwbf.fwbf_decode_batch(batch)
    torch.cuda.synchronize()
    fwbf.fwbf_batch_destroy(batch)
    for j, (b, it) in zip(jobs, outs):
        idx = np.arange(0, j["q"].shape[0], 11)[:12]
        bo, io = oracle.fwbf_i8(j["h"], j["p"], j["q"][idx], 60, alpha=1.5)
        assert np.array_equal(it.cpu().numpy()[idx], io), j["key"]
        assert np.array_equal(b.cpu().numpy().view(np.uint32)[idx], bo), j["key"]


def test_batch_graph_replay(fwbf, jobs):
    outs = [j["code"].outputs(j["qd"].shape[0]) for j in jobs]
    spec = [(j["code"].handle, j["qd"], 60, 1.5, b, it) for j, (b, it) in zip(jobs, outs)]
    batch = fwbf.fwbf_batch_create(spec)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fwbf.fwbf_decode_batch(batch, s)  # warm-up outside capture
    torch.cuda.synchronize()
    ref = [(b.clone(), it.clone()) for b, it in outs]
    for b, it in outs:
        b.fill_(-1)
        it.fill_(-99)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fwbf.fwbf_decode_batch(batch, s)
    for _ in range(2):
        for b, it in outs:
            b.fill_(-1)
            it.fill_(-99)
        g.replay()
        torch.cuda.synchronize()
        for (b, it), (rb, ri) in zip(outs, ref):
            assert torch.equal(b, rb) and torch.equal(it, ri)
    fwbf.fwbf_batch_destroy(batch)
