"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

int8 path: decisions and pass counts bit-exact on every frame.  float32 path:
first-pass metric within 1e-5 relative to the magnitude of its terms, and
decisions identical on every frame whose decision margins exceed that bound.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1206_3362_gb300.inputs import Encoder, bpsk_awgn, make_code, random_codewords

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def fwbf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1206_3362_gb300 import fwbf as mod

    return mod


def gpu_decode(fwbf, h, p, q, max_iter, alpha):
    with fwbf.Code.from_parity_check(h, p) as code:
        qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
        bits, iters = code.decode(qd, max_iter, alpha)
        torch.cuda.synchronize()
        assert fwbf.fwbf_last_status() == 0
        return bits.cpu().numpy().view(np.uint32), iters.cpu().numpy()


def frames(key, F, ebn0, seed, zero=False):
    h = make_code(key)
    enc = Encoder(h)
    if zero:
        c = np.zeros((F, h.N), dtype=np.uint8)
    else:
        _, c = random_codewords(enc, F, seed=seed)
    y = bpsk_awgn(c, ebn0, enc.rate, seed=seed)
    return h, c, y


def assert_same(fwbf, h, p, q, max_iter, alpha, threads=None):
    b_gpu, i_gpu = gpu_decode(fwbf, h, p, q, max_iter, alpha)
    b_ref, i_ref, _ = oracle.fwbf_i8_threaded(h, p, q, max_iter, alpha, threads=threads)
    bad = np.flatnonzero((i_gpu != i_ref) | (b_gpu != b_ref).any(axis=1))
    assert bad.size == 0, f"{bad.size} frames differ, first {bad[:5]}: gpu {i_gpu[bad[:5]]} oracle {i_ref[bad[:5]]}"
    return i_ref


# ---------------------------------------------------------------------------
# quantiser
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("count,offset", [(0, 0), (1, 0), (3, 1), (4097, 0), (4097, 3), (1 << 20, 0)])
def test_quantize_matches_oracle(fwbf, count, offset):
    rng = np.random.default_rng(count + offset)
    y = (rng.standard_normal(count + offset) * 4).astype(np.float32)
    special = np.array([0.0, -0.0, 1 / 32, -1 / 32, 3 / 32, 5 / 32, 7.96875, 8.0, -8.0, 1e30,
                        np.nan, np.inf, -np.inf, -1e-40], dtype=np.float32)
    y[: min(y.size, special.size)] = special[: min(y.size, special.size)]
    yd = torch.from_numpy(y).cuda()[offset:]
    q = torch.empty(count, dtype=torch.int8, device="cuda")
    fwbf.fwbf_quantize(yd, q)
    torch.cuda.synchronize()
    assert np.array_equal(q.cpu().numpy(), oracle.quantize(y[offset:]))


# ---------------------------------------------------------------------------
# int8 decoder, bit-exact
# ---------------------------------------------------------------------------

def test_small_random_code_workload(fwbf):
    """(3,6)-regular N=504, all-zero codeword, 4 dB, 1000 frames, K_max = 50,
    p = 32 (ragged last block of 24)."""
    h, c, y = frames("rand504", 1000, 4.0, seed=1, zero=True)
    q = oracle.quantize(y)
    assert_same(fwbf, h, 32, q, 50, 1.5)


@pytest.mark.parametrize("ebn0", [3.0, 4.0, 5.0])
@pytest.mark.parametrize("p", [31, 93])
def test_eg1023(fwbf, ebn0, p):
    h, c, y = frames("eg1023", 384, ebn0, seed=3)
    assert_same(fwbf, h, p, oracle.quantize(y), 100, 1.5)


@pytest.mark.parametrize("p", [1, 16, 100, 255])
@pytest.mark.parametrize("max_iter", [1, 5, 10, 50])
def test_eg255_block_lengths_and_kmax(fwbf, p, max_iter):
    h, c, y = frames("eg255", 300, 3.0, seed=p * 100 + max_iter)
    assert_same(fwbf, h, p, oracle.quantize(y), max_iter, 1.0)


@pytest.mark.parametrize("key,p", [("rand2016", 32), ("qc8192", 64), ("eg4095", 63)])
def test_other_codes(fwbf, key, p):
    h, c, y = frames(key, 64, 4.0, seed=5)
    assert_same(fwbf, h, p, oracle.quantize(y), 30, 1.5)


def test_generic_kernel_warp_groups(fwbf):
    """Codes whose frames fill a block's shared memory run several warps per
    frame in the list decoder: the QC N = 16384 code with its columns permuted
    (no circulant structure left; 8 warps, wide rows: a check's edges shared by
    the lanes) and a random (3,6) N = 8064 code (narrow rows: a lane per
    syndrome word), both against the oracle, with a ragged tail."""
    from paper_1206_3362_gb300.inputs.codes import ParityCheck, random_regular

    h0, c, y = frames("qc16384", 37, 5.5, seed=61)
    perm = np.random.default_rng(1).permutation(h0.N)
    h = ParityCheck(N=h0.N, M=h0.M, rows=h0.rows, cols=perm[h0.cols].astype(np.int32))
    yp = np.empty_like(y)
    yp[:, perm] = y
    with fwbf.Code.from_parity_check(h, 32) as code:
        assert code.info.Z == 1 and code.info.decoder == fwbf.FWBF_DECODER_LIST
    assert_same(fwbf, h, 32, oracle.quantize(yp), 30, 1.5)
    h = random_regular(8064, 3, 6, seed=62)
    enc = Encoder(h)
    _, c = random_codewords(enc, 45, seed=63)
    assert_same(fwbf, h, 32, oracle.quantize(bpsk_awgn(c, 6.0, enc.rate, seed=63)), 40, 1.0)


def test_generic_kernel_on_permuted_eg1023(fwbf):
    """The same EG(1023,781) code with its columns permuted has no circulant
    structure, so it runs through the generic (list-based) kernel instead of
    the packed cyclic one; both must match the oracle."""
    from paper_1206_3362_gb300.inputs.codes import ParityCheck

    h0, c, y = frames("eg1023", 256, 3.5, seed=31)
    perm = np.random.default_rng(0).permutation(h0.N)
    h = ParityCheck(N=h0.N, M=h0.M, rows=h0.rows, cols=perm[h0.cols].astype(np.int32))
    yp = np.empty_like(y)
    yp[:, perm] = y
    with fwbf.Code.from_parity_check(h, 31) as code:
        assert code.info.Z == 1
    assert_same(fwbf, h, 31, oracle.quantize(yp), 100, 1.5)


def test_circulant_structure_detected(fwbf):
    for key, Z, dec in (("eg1023", 1023, fwbf.FWBF_DECODER_CYCLIC), ("qc8192", 256, fwbf.FWBF_DECODER_QC),
                        ("qc16384", 512, fwbf.FWBF_DECODER_QC), ("rand504", 1, fwbf.FWBF_DECODER_LIST)):
        h = make_code(key)
        with fwbf.Code.from_parity_check(h, 31) as code:
            assert code.info.Z == Z
            assert code.info.decoder == dec


def _qc_from_weights(Z, base, seed):
    """H of Z x Z blocks, block (r, c) the sum of base[r][c] distinct seeded
    circulant permutations (0: an all-zero block)."""
    from paper_1206_3362_gb300.inputs.codes import quasi_cyclic

    rng = np.random.default_rng(seed)
    return quasi_cyclic(Z, [[sorted(rng.choice(Z, size=w, replace=False).tolist()) for w in row] for row in base])


def _qc_random_weights(MB, NB, seed):
    """Irregular base matrix: block weights drawn from {0, 1, 1, 1, 2}, every
    block row of weight >= 2."""
    rng = np.random.default_rng(seed)
    base = rng.choice([0, 1, 1, 1, 2], size=(MB, NB))
    for r in range(MB):
        while base[r].sum() < 2:
            base[r, rng.integers(NB)] = 1
    return base.tolist()


# Quasi-cyclic codes the packed QC decoder takes, chosen to reach each of its
# forms: R = 8, 4, 2, 1 pairs per lane per gather chunk (Z / 64 divisible by 8,
# 4, 2, odd) and 1, 4 or 8 warps per frame (frames per block 24, 5-6, 2), with
# irregular column weights, all-zero blocks, blocks of two circulants and an
# all-zero block column (bits in no check).
_QC_CASES = {
    "z64_empty_col": (64, [[1, 1, 0, 2, 1, 1, 0, 1, 0], [0, 1, 1, 1, 2, 0, 1, 1, 0],
                           [1, 0, 1, 1, 0, 1, 1, 1, 0]]),
    "z128_weight2": (128, [[2, 1, 0, 1, 2, 1], [1, 2, 1, 1, 0, 2]]),
    "z256_irregular": (256, "3x6"),
    "z320_irregular": (320, "2x5"),
    "z512_wpf2": (512, "3x8"),
    "z192_wpf4": (192, "5x40"),
    "z576_wpf8": (576, "4x40"),
}


@pytest.mark.parametrize("case", sorted(_QC_CASES))
def test_qc_packed_decoder(fwbf, case):
    """The packed quasi-cyclic decoder against the oracle, bit-exact: all-zero
    codeword under AWGN at 5.5, 6.5 and 7.5 dB (a third of the frames each:
    frames that converge, frames that stall; valid for any H), several block
    lengths p (1 or 4, a ragged one, N), K_max 1 and 40, alpha 0 and 1.5."""
    Z, base = _QC_CASES[case]
    seed = Z + len(case)
    if isinstance(base, str):
        MB, NB = map(int, base.split("x"))
        base = _qc_random_weights(MB, NB, seed)
    h = _qc_from_weights(Z, base, seed)
    F = 11 if h.N > 10000 else 29
    rate = max(0.3, 1.0 - h.M / h.N)
    parts = np.array_split(np.zeros((F, h.N), dtype=np.uint8), 3)
    y = np.concatenate([bpsk_awgn(c, e, rate, seed=seed) for c, e in zip(parts, (5.5, 6.5, 7.5))])
    q = oracle.quantize(y)
    p_small = 1 if h.N <= 8192 else 4  # p = 1 at N = 23040: 8 N bytes of block keys do not fit
    for p, max_iter, alpha in ((37, 40, 1.5), (p_small, 1, 1.5), (h.N, 40, 0.0), (64, 40, 1.5)):
        with fwbf.Code.from_parity_check(h, p) as code:
            assert code.info.Z == Z and code.info.decoder == fwbf.FWBF_DECODER_QC
        assert_same(fwbf, h, p, q, max_iter, alpha)


@pytest.mark.parametrize("alpha", [0.0, 0.5, 3.0, 63.75])
def test_alpha_range(fwbf, alpha):
    h, c, y = frames("eg255", 200, 3.5, seed=8)
    assert_same(fwbf, h, 16, oracle.quantize(y), 20, alpha)


def test_edge_frames(fwbf):
    """Saturated values, zeros, constant magnitudes (every metric tie), and
    frames that never converge."""
    h = make_code("eg255")
    rng = np.random.default_rng(0)
    q = []
    q.append(np.full(h.N, 127, dtype=np.int8))
    q.append(np.full(h.N, -127, dtype=np.int8))
    q.append(np.zeros(h.N, dtype=np.int8))
    q.append(np.where(rng.random(h.N) < 0.5, 16, -16).astype(np.int8))        # heavy ties
    q.append(np.where(rng.random(h.N) < 0.1, -127, 127).astype(np.int8))
    q.append(rng.integers(-127, 128, h.N).astype(np.int8))                     # noise only
    q.append(rng.integers(-2, 3, h.N).astype(np.int8))                         # tiny magnitudes
    for _ in range(25):
        q.append(rng.integers(-127, 128, h.N).astype(np.int8))
    q = np.stack(q)
    for p in (1, 5, 255):
        i = assert_same(fwbf, h, p, q, 25, 1.0)
    assert (i < 0).any()


@pytest.mark.parametrize("key,p", [("eg255", 16), ("rand504", 32), ("qc8192", 64)])
def test_minus_128_reads_as_minus_127(fwbf, key, p):
    """int8 inputs of -128 (outside the quantiser's range) decode as -127 in
    every decoder (cyclic, list, quasi-cyclic), as the oracle reads them."""
    h, c, y = frames(key, 24, 3.5, seed=14, zero=True)
    q = oracle.quantize(y)
    rng = np.random.default_rng(15)
    q[rng.random(q.shape) < 0.05] = -128
    q[0, :] = -128
    i = assert_same(fwbf, h, p, q, 20, 1.5)
    q127 = np.maximum(q, -127).astype(np.int8)
    assert np.array_equal(i, assert_same(fwbf, h, p, q127, 20, 1.5))


def test_frame_counts_ragged(fwbf):
    """n_frames 0, 1 and counts that leave warps, CTAs and the last 16-byte
    chunk of the buffer partly filled."""
    h, c, y = frames("rand504", 777, 3.0, seed=12)
    q = oracle.quantize(y)
    for F in (1, 2, 33, 777):
        assert_same(fwbf, h, 32, q[:F], 20, 1.5)
    with fwbf.Code.from_parity_check(h, 32) as code:
        bits, iters = code.outputs(0)
        fwbf.fwbf_decode(code.handle, torch.empty((0, h.N), dtype=torch.int8, device="cuda"), 20, 1.5, bits, iters)
        torch.cuda.synchronize()


def test_odd_length_frames_unaligned_offsets(fwbf):
    """N = 255 bytes per frame: every frame starts at a different offset inside
    its 16-byte chunk."""
    h, c, y = frames("eg255", 257, 3.0, seed=13)
    assert_same(fwbf, h, 16, oracle.quantize(y), 15, 1.0)


def test_all_weight_two_errors_eg15(fwbf):
    """Brute force on the (15,7) code: every error pattern of weight <= 2 on a
    noiseless frame, for every block length."""
    h = make_code("eg15")
    pats = [()] + [(i,) for i in range(15)] + [(i, j) for i in range(15) for j in range(i + 1, 15)]
    q = np.full((len(pats), 15), 16, dtype=np.int8)
    for f, pat in enumerate(pats):
        q[f, list(pat)] = -16
    for p in range(1, 16):
        i = assert_same(fwbf, h, p, q, 10, 1.0)
        assert (i >= 0).all()


def test_hand_traced_frame(fwbf):
    with open(os.path.join(GOLD, "eg15_trace.json")) as f:
        g = json.load(f)
    h = make_code("eg15")
    q = np.array(g["q"], dtype=np.int8)[None]
    bits, iters = gpu_decode(fwbf, h, g["p"], q, g["max_iter"], g["alpha"])
    assert iters[0] == g["iters"]
    assert oracle.unpack_bits(bits, 15)[0].tolist() == g["z"]


def test_full_size_sampled(fwbf):
    """EG(1023,781) at 4 dB with 2^18 frames in one launch; 512 sampled frames
    checked against the oracle, and every converged frame checks H z = 0."""
    h = make_code("eg1023")
    enc = Encoder(h)
    from paper_1206_3362_gb300.inputs.channel import bpsk_awgn_torch, random_codewords_torch

    F = 1 << 18
    _, c = random_codewords_torch(enc, F, seed=5, device="cuda")
    y = bpsk_awgn_torch(c, 4.0, enc.rate, seed=5)
    with fwbf.Code.from_parity_check(h, 31) as code:
        q = fwbf.quantize(y)
        bits, iters = code.decode(q, 100, 1.5)
        torch.cuda.synchronize()
    idx = np.random.default_rng(1).choice(F, 512, replace=False)
    qs = q[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert np.array_equal(qs, oracle.quantize(y[torch.from_numpy(idx).cuda()].cpu().numpy()))
    bo, io, _ = oracle.fwbf_i8_threaded(h, 31, qs, 100, 1.5)
    assert np.array_equal(iters.cpu().numpy()[idx], io)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32)[idx], bo)
    # every converged frame is a codeword (syndrome computed with torch on the device)
    zb = bits.view(torch.uint8)  # little-endian: byte k holds bits 8k..8k+7
    z = ((zb.unsqueeze(-1) >> torch.arange(8, device="cuda", dtype=torch.uint8)) & 1).reshape(F, -1)[:, :h.N]
    Hd = torch.zeros((h.M, h.N), dtype=torch.float32, device="cuda")
    Hd[torch.from_numpy(h.rows.astype(np.int64)).cuda(), torch.from_numpy(h.cols.astype(np.int64)).cuda()] = 1
    syn = (z[:65536].float() @ Hd.T).to(torch.int64) % 2
    conv = iters[:65536] >= 0
    assert not syn[conv].any() and syn[~conv].any(dim=1).all()


# ---------------------------------------------------------------------------
# float32 decoder against the float64 oracle
# ---------------------------------------------------------------------------

def _term_scale(h, y, alpha):
    """sum_m w_{n,m} + alpha |y_n| per bit: the size of the terms of Eq. 1."""
    a = np.abs(y.astype(np.float64))
    csr = h.csr()
    scale = np.zeros_like(a)
    for m in range(h.M):
        bits = csr.indices[csr.indptr[m]:csr.indptr[m + 1]]
        v = a[:, bits]
        order = np.sort(v, axis=1)
        m1, m2 = order[:, :1], order[:, 1:2]
        w = np.where(v == m1, m2, m1)
        scale[:, bits] += w
    return scale + alpha * a


@pytest.mark.parametrize("key,p", [("eg1023", 31), ("rand504", 32)])
def test_f32_first_metric(fwbf, key, p):
    h, c, y = frames(key, 64, 3.5, seed=21)
    with fwbf.Code.from_parity_check(h, p) as code:
        E = code.metric_f32(torch.from_numpy(y).cuda(), 1.5).cpu().numpy()
    _, _, _, e0 = oracle.fwbf_f64(h, p, y, 1, alpha=1.5, want_E0=True)
    tol = 1e-5 * _term_scale(h, y, 1.5)
    assert np.all(np.abs(E - e0) <= tol)


@pytest.mark.parametrize("key,p,ebn0", [("eg1023", 31, 3.5), ("eg1023", 93, 4.0), ("rand504", 32, 3.0)])
def test_f32_decisions(fwbf, key, p, ebn0):
    h, c, y = frames(key, 256, ebn0, seed=22)
    with fwbf.Code.from_parity_check(h, p) as code:
        bits, iters = code.decode_f32(torch.from_numpy(y).cuda(), 100, 1.5)
        bits = bits.cpu().numpy().view(np.uint32)
        iters = iters.cpu().numpy()
    bo, io, margin = oracle.fwbf_f64(h, p, y, 100, alpha=1.5)
    tol = 1e-5 * _term_scale(h, y, 1.5).max(axis=1)
    clear = margin > 2 * tol
    same = (iters == io) & (bits == bo).all(axis=1)
    assert same[clear].all()
    assert clear.mean() > 0.9, f"near-tie frames: {(~clear).sum()}"


# ---------------------------------------------------------------------------
# lambda-largest selection (comparison rule) against the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("key,lam", [("eg255", 1), ("eg255", 10), ("eg1023", 10), ("eg1023", 3),
                                     ("rand504", 64), ("eg255", 255)])
def test_lambda_selection_matches_oracle(fwbf, key, lam):
    h, c, y = frames(key, 160, 3.25, seed=60 + lam)
    q = oracle.quantize(y)
    with fwbf.Code.from_parity_check(h, 31 if h.N > 31 else 5) as code:
        bits, iters = code.outputs(160)
        fwbf.fwbf_decode_lambda(code.handle, torch.from_numpy(q).cuda(), 30, 1.5, lam, bits, iters)
        torch.cuda.synchronize()
    bo, io = oracle.lambda_i8(h, lam, q, 30, alpha=1.5)
    assert np.array_equal(iters.cpu().numpy(), io)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), bo)


def test_decode_host_pipeline(fwbf):
    """Host float frames in, host decisions out, in chunks over two streams:
    identical to quantise + decode on the device, for chunk sizes that divide
    the batch and that leave a ragged last chunk."""
    h, c, y = frames("eg1023", 1000, 3.75, seed=71)
    q = oracle.quantize(y)
    bo, io, _ = oracle.fwbf_i8_threaded(h, 31, q, 100, 1.5)
    with fwbf.Code.from_parity_check(h, 31) as code:
        for chunk in (1000, 256, 333, 1):
            yh = torch.from_numpy(y).pin_memory() if chunk != 333 else torch.from_numpy(y)
            bh = torch.zeros((1000, code.words), dtype=torch.int32)
            ih = torch.zeros(1000, dtype=torch.int32)
            fwbf.fwbf_decode_host(code.handle, yh, 100, 1.5, bh, ih, chunk_frames=chunk)
            torch.cuda.synchronize()
            assert np.array_equal(ih.numpy(), io), chunk
            assert np.array_equal(bh.numpy().view(np.uint32), bo), chunk


def test_zero_frames_every_entry_point(fwbf):
    """n_frames = 0 is a no-op for every decoding entry point and for a batch
    job, and leaves the status clean."""
    from paper_1206_3362_gb300.learned import Network

    h = make_code("eg255")
    net = Network(seed=1)
    with fwbf.Code.from_parity_check(h, 16) as code:
        q0 = torch.empty((0, h.N), dtype=torch.int8, device="cuda")
        y0 = torch.empty((0, h.N), dtype=torch.float32, device="cuda")
        bits, iters = code.outputs(0)
        fwbf.fwbf_decode(code.handle, q0, 10, 1.5, bits, iters)
        fwbf.fwbf_decode_noalloc(code.handle, q0, 10, 1.5, bits, iters)
        fwbf.fwbf_decode_f32(code.handle, y0, 10, 1.5, bits, iters)
        fwbf.fwbf_decode_lambda(code.handle, q0, 10, 1.5, 4, bits, iters)
        a0 = torch.empty((0, 10), dtype=torch.int32, device="cuda")
        fwbf.fwbf_decode_sched(code.handle, q0, 10, a0, a0, bits, iters)
        fwbf.fwbf_decode_learned(code.handle, q0, 10, 4, 1.5, net.blob, bits, iters)
        fwbf.fwbf_decode_host(code.handle, torch.empty((0, h.N), dtype=torch.float32), 10, 1.5,
                              torch.empty((0, code.words), dtype=torch.int32), torch.empty(0, dtype=torch.int32))
        h2, c2, y2 = frames("eg255", 3, 4.0, seed=2)
        q2 = torch.from_numpy(oracle.quantize(y2)).cuda()
        b2, i2 = code.outputs(3)
        batch = fwbf.fwbf_batch_create([(code.handle, q0, 10, 1.5, bits, iters), (code.handle, q2, 10, 1.5, b2, i2)])
        try:
            fwbf.fwbf_decode_batch(batch)
            torch.cuda.synchronize()
            assert fwbf.fwbf_batch_status() == 0
        finally:
            fwbf.fwbf_batch_destroy(batch)
        bo, io = oracle.fwbf_i8(h, 16, oracle.quantize(y2), 10, 1.5)
        assert np.array_equal(i2.cpu().numpy(), io)
        torch.cuda.synchronize()
        assert fwbf.fwbf_last_status() == 0


def test_code_beyond_shared_memory_is_rejected(fwbf):
    """A code whose frame state does not fit one block's shared memory (random
    (3,6) N = 40,000: ~290 KB per frame) is rejected with FWBF_EUNSUPPORTED
    before anything is launched; the next call decodes normally."""
    from paper_1206_3362_gb300.inputs.codes import random_regular

    h = random_regular(40000, 3, 6, seed=64)
    with fwbf.Code.from_parity_check(h, 32) as code:
        q = torch.zeros((2, h.N), dtype=torch.int8, device="cuda")
        bits, iters = code.outputs(2)
        with pytest.raises(fwbf.FwbfError) as err:
            fwbf.fwbf_decode(code.handle, q, 10, 1.5, bits, iters)
        assert err.value.status == fwbf.FWBF_EUNSUPPORTED
    h, c, y = frames("eg255", 20, 4.0, seed=65)
    assert_same(fwbf, h, 16, oracle.quantize(y), 10, 1.5)


def test_rc_constraint_reported(fwbf):
    """fwbf_code_info.max_row_overlap: 1 for the EG and QC codes (any two lines
    of a Euclidean geometry meet in at most one point), at most 1 for the
    4-cycle-free random code, 2 for an H with a 4-cycle (warned, or rejected on
    request); the decoder still matches the oracle on that H."""
    import warnings

    from paper_1206_3362_gb300.inputs.codes import ParityCheck

    for key in ("eg255", "eg1023", "qc8192"):
        with fwbf.Code.from_parity_check(make_code(key), 16) as code:
            assert code.info.max_row_overlap == 1, key
    with fwbf.Code.from_parity_check(make_code("rand504"), 32) as code:
        assert code.info.max_row_overlap <= 1
    # checks 0 and 1 share bits 0 and 1
    rows = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3], dtype=np.int32)
    cols = np.array([0, 1, 2, 0, 1, 3, 2, 4, 5, 3, 4, 5], dtype=np.int32)
    h = ParityCheck(N=6, M=4, rows=rows, cols=cols)
    with warnings.catch_warnings(record=True) as w:
        warnings.simplefilter("always")
        code = fwbf.Code.from_parity_check(h, 2)
    assert code.info.max_row_overlap == 2 and any("RC constraint" in str(x.message) for x in w)
    q = np.array([[10, -3, 7, 20, -5, 9], [-12, -12, 4, 4, 4, -4]], dtype=np.int8)
    bits, iters = code.decode(torch.from_numpy(q).cuda(), 8, 1.0)
    torch.cuda.synchronize()
    code.close()
    bo, io = oracle.fwbf_i8(h, 2, q, 8, 1.0)
    assert np.array_equal(iters.cpu().numpy(), io) and np.array_equal(bits.cpu().numpy().view(np.uint32), bo)
    with pytest.raises(ValueError):
        fwbf.Code.from_parity_check(h, 2, require_rc=True)
