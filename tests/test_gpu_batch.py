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


def _qc_irregular(Z, MB, NB, seed):
    """Seeded QC code with block weights from {0, 1, 1, 1, 2} (irregular
    column weights, all-zero blocks, blocks of two circulants)."""
    from paper_1206_3362_gb300.inputs.codes import quasi_cyclic

    rng = np.random.default_rng(seed)
    base = rng.choice([0, 1, 1, 1, 2], size=(MB, NB))
    for r in range(MB):
        while base[r].sum() < 2:
            base[r, rng.integers(NB)] = 1
    return quasi_cyclic(Z, [[sorted(rng.choice(Z, size=int(w), replace=False).tolist()) for w in row]
                            for row in base])


@pytest.mark.parametrize("warps,packed", [(16, 2), (16, 1), (8, 1), (4, 1)])
def test_batch_quasi_cyclic_jobs(fwbf, warps, packed):
    """QC jobs in the packed batch: QC N=16384 (Z=512, one to three frames per
    CTA, groups of 8 warps), an irregular Z=256 code (groups of 4) and a Z=192
    code (list decoder), beside EG(255); every job equals fwbf_decode, and
    sampled frames equal the oracle."""
    specs = [(make_code("qc16384"), 32, 23), (_qc_irregular(256, 3, 8, seed=71), 37, 41),
             (_qc_irregular(192, 3, 9, seed=72), 32, 33), (make_code("eg255"), 16, 50)]
    jobs = []
    try:
        for i, (h, p, F) in enumerate(specs):
            parts = np.array_split(np.zeros((F, h.N), dtype=np.uint8), 3)
            rate = max(0.3, 1.0 - h.M / h.N)
            y = np.concatenate([bpsk_awgn(c, e, rate, seed=80 + i) for c, e in zip(parts, (5.5, 6.5, 7.5))])
            q = oracle.quantize(y)
            jobs.append(dict(h=h, p=p, q=q, qd=torch.from_numpy(q).cuda(), code=fwbf.Code.from_parity_check(h, p)))
        assert [j["code"].info.decoder for j in jobs] == [fwbf.FWBF_DECODER_QC] * 3 + [fwbf.FWBF_DECODER_CYCLIC]
        outs = [j["code"].outputs(j["qd"].shape[0]) for j in jobs]
        spec = [(j["code"].handle, j["qd"], 40, 1.5, b, it) for j, (b, it) in zip(jobs, outs)]
        batch = fwbf.fwbf_batch_create(spec, warps_per_cta=warps, packed=packed)
        try:
            info = [fwbf.fwbf_batch_query(batch, k) for k in range(len(spec))]
            # EG(255) (H / 32 = 4) keeps the grouped kernel out; the mixed kernel
            # never gives a job 16 warps per frame (it would skip such a job)
            assert not any(i.grouped for i in info)
            assert all(i.warps_per_frame in (1, 2, 4, 8) for i in info)
            assert [i.decoder for i in info] == [fwbf.FWBF_DECODER_QC, fwbf.FWBF_DECODER_QC, fwbf.FWBF_DECODER_LIST,
                                                 fwbf.FWBF_DECODER_CYCLIC]
            fwbf.fwbf_decode_batch(batch)
            torch.cuda.synchronize()
            assert fwbf.fwbf_batch_status() == 0
        finally:
            fwbf.fwbf_batch_destroy(batch)
        for k, (j, (b, it)) in enumerate(zip(jobs, outs)):
            sb, si = j["code"].decode(j["qd"], 40, 1.5)
            torch.cuda.synchronize()
            assert np.array_equal(it.cpu().numpy(), si.cpu().numpy()), k
            assert np.array_equal(b.cpu().numpy(), sb.cpu().numpy()), k
            idx = np.arange(0, j["q"].shape[0], 5)[:8]
            bo, io = oracle.fwbf_i8(j["h"], j["p"], j["q"][idx], 40, alpha=1.5)
            assert np.array_equal(it.cpu().numpy()[idx], io), k
            assert np.array_equal(b.cpu().numpy().view(np.uint32)[idx], bo), k
    finally:
        for j in jobs:
            j["code"].close()


def test_batch_grouped_qc_frame_fills_block(fwbf):
    """The grouped kernel with a QC N=16384 job: one of its frames fills a
    block's shared memory, so all 16 warps of the block decode it; beside an
    EG(1023,781) job (two warps per frame).  Both jobs equal fwbf_decode."""
    specs = [(make_code("qc16384"), 32, 40, 5.5), (make_code("eg1023"), 31, 96, 3.5)]
    jobs = []
    try:
        for i, (h, p, F, eb) in enumerate(specs):
            c = np.zeros((F, h.N), dtype=np.uint8)
            q = oracle.quantize(bpsk_awgn(c, eb, max(0.5, 1.0 - h.M / h.N), seed=90 + i))
            jobs.append(dict(qd=torch.from_numpy(q).cuda(), code=fwbf.Code.from_parity_check(h, p)))
        outs = [j["code"].outputs(j["qd"].shape[0]) for j in jobs]
        spec = [(j["code"].handle, j["qd"], 40, 1.5, b, it) for j, (b, it) in zip(jobs, outs)]
        batch = fwbf.fwbf_batch_create(spec, warps_per_cta=16, packed=2)
        try:
            qc, eg = fwbf.fwbf_batch_query(batch, 0), fwbf.fwbf_batch_query(batch, 1)
            assert qc.grouped == 1 and eg.grouped == 1
            assert (qc.decoder, qc.warps_per_frame, qc.frames_per_cta) == (fwbf.FWBF_DECODER_QC, 16, 1)
            assert (eg.decoder, eg.warps_per_frame) == (fwbf.FWBF_DECODER_CYCLIC, 2)
            fwbf.fwbf_decode_batch(batch)
            torch.cuda.synchronize()
            assert fwbf.fwbf_batch_status() == 0
        finally:
            fwbf.fwbf_batch_destroy(batch)
        for k, (j, (b, it)) in enumerate(zip(jobs, outs)):
            sb, si = j["code"].decode(j["qd"], 40, 1.5)
            torch.cuda.synchronize()
            assert torch.equal(it, si) and torch.equal(b, sb), k
    finally:
        for j in jobs:
            j["code"].close()
