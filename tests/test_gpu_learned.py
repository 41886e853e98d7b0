"""GPU checks of the per-pass schedule, the learned schedule and the network
kernels: scheduled decoding bit-exact against the oracle, features against
values derived from the oracle's trace, learned decoding replayed exactly by
the oracle from the schedule it recorded, network forward/gradient/Adam
against the float64 reference, and what a trained network gains over plain
FWBF."""
import numpy as np
import pytest

import oracle
from oracle import mlp as mlp_ref
from paper_1206_3362_gb300.inputs import Encoder, bpsk_awgn, make_code, random_codewords

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


def frames(key, F, ebn0, seed):
    h = make_code(key)
    enc = Encoder(h)
    _, c = random_codewords(enc, F, seed=seed)
    return h, c, oracle.quantize(bpsk_awgn(c, ebn0, enc.rate, seed=seed))


# ---------------------------------------------------------------------------
# network kernels against the float64 reference
# ---------------------------------------------------------------------------

def _master(seed, scale=0.2):
    return (np.random.default_rng(seed).standard_normal(mlp_ref.N_PARAMS) * scale).astype(np.float32)


def test_mlp_forward(fwbf):
    master = _master(1)
    x = np.random.default_rng(2).standard_normal((333, 8)).astype(np.float32)
    blob = torch.zeros(fwbf.MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
    fwbf.fwbf_mlp_pack(torch.from_numpy(master).cuda(), blob)
    out = torch.empty((333, 2), device="cuda")
    fwbf.fwbf_mlp_forward(blob, torch.from_numpy(x).cuda(), out)
    ref, _ = mlp_ref.forward(master, x)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)


def test_mlp_gradient(fwbf):
    master = _master(3)
    rng = np.random.default_rng(4)
    n = 100  # not a multiple of the kernel's 32-sample blocks
    x = rng.standard_normal((n, 8)).astype(np.float32)
    t = rng.standard_normal((n, 2)).astype(np.float32)
    blob = torch.zeros(fwbf.MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
    fwbf.fwbf_mlp_pack(torch.from_numpy(master).cuda(), blob)
    grad = torch.zeros(fwbf.MLP_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    fwbf.fwbf_mlp_grad(blob, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), n, grad, loss)
    ref_loss, ref_g = mlp_ref.loss_and_grad(master, x, t)
    g = grad.cpu().numpy()
    assert abs(loss.item() - ref_loss) <= 1e-4 * abs(ref_loss)
    scale = np.abs(ref_g).max()
    assert np.allclose(g, ref_g, rtol=1e-3, atol=1e-5 * scale)


def test_mlp_adam_step(fwbf):
    master = _master(5)
    g = (np.random.default_rng(6).standard_normal(mlp_ref.N_PARAMS) * 0.1).astype(np.float32)
    dm = torch.from_numpy(master).cuda()
    blob = torch.zeros(fwbf.MLP_BLOB_BYTES, dtype=torch.uint8, device="cuda")
    m = torch.zeros(fwbf.MLP_PARAMS, device="cuda")
    v = torch.zeros_like(m)
    grad = torch.from_numpy(g).cuda()
    fwbf.fwbf_mlp_adam(dm, blob, grad, m, v, 1, 1e-3)
    ref, _, _ = mlp_ref.adam_step(master.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, 1e-3)
    assert np.allclose(dm.cpu().numpy(), ref, atol=2e-6)
    assert not grad.any()
    w = blob[:9472].view(torch.int16).cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    assert np.array_equal(w.view(np.float32), mlp_ref.bf16_round(dm.cpu().numpy()[:4736]).astype(np.float32))


# ---------------------------------------------------------------------------
# per-pass schedules
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("key,p", [("eg255", 16), ("eg1023", 8), ("eg1023", 31)])
def test_decode_sched_matches_oracle(fwbf, key, p):
    h, c, q = frames(key, 160, 3.0, seed=41)
    K = 25
    rng = np.random.default_rng(42)
    A = rng.integers(0, 900, size=(160, K)).astype(np.int32)
    T = (rng.integers(0, 4, size=(160, K)) * 512).astype(np.int32)
    with fwbf.Code.from_parity_check(h, p) as code:
        bits, iters = code.outputs(160)
        fwbf.fwbf_decode_sched(code.handle, torch.from_numpy(q).cuda(), K, torch.from_numpy(A).cuda(),
                               torch.from_numpy(T).cuda(), bits, iters)
        torch.cuda.synchronize()
    bo, io = oracle.fwbf_i8(h, p, q, K, alpha_sched=A, theta_sched=T)
    assert np.array_equal(iters.cpu().numpy(), io)
    assert np.array_equal(bits.cpu().numpy().view(np.uint32), bo)


def test_features_match_oracle_trace(fwbf):
    h, c, q = frames("eg255", 12, 2.5, seed=43)
    K, P = 10, 6
    A = np.full((12, K), 384, dtype=np.int32)
    T = np.zeros((12, K), dtype=np.int32)
    with fwbf.Code.from_parity_check(h, 16) as code:
        bits, iters = code.outputs(12)
        feat = torch.full((12, P, 8), -1.0, device="cuda")
        fwbf.fwbf_decode_sched(code.handle, torch.from_numpy(q).cuda(), K, torch.from_numpy(A).cuda(),
                               torch.from_numpy(T).cuda(), bits, iters, out_feat=feat)
        torch.cuda.synchronize()
        B = code.info.n_blocks
    feat = feat.cpu().numpy()
    a = np.abs(q.astype(np.int64))
    for f in range(12):
        _, it, tr = oracle.fwbf_i8(h, 16, q[f:f + 1], K, alpha=1.5, trace=True)
        passes = it[0] if it[0] >= 0 else K
        W = tr["s"].sum(axis=1)
        for k in range(min(passes, P)):
            D_prev = (tr["E"][k - 1] + 384 * a[f]) // 256 if k > 0 else None
            want = [W[k] / h.N, (W[k - 1] if k else W[0]) / h.N, W[0] / h.N, k / 16.0,
                    (tr["flip"][k - 1].sum() / B) if k else 0.0,
                    ((D_prev >= 1).sum() / h.N) if k else 0.0,
                    a[f].sum() / (127.0 * h.N), (a[f] < 8).sum() / h.N]
            assert np.allclose(feat[f, k], want, rtol=1e-6, atol=1e-7), (f, k, feat[f, k], want)


# ---------------------------------------------------------------------------
# learned schedule
# ---------------------------------------------------------------------------

def _varied_network():
    from paper_1206_3362_gb300.learned import Network

    net = Network(seed=7)
    m = net.master.cpu().numpy()
    rng = np.random.default_rng(8)
    m[4608:4736] = rng.standard_normal(128) * 0.3   # W3: outputs vary with the features
    m[4864:4866] = [1.5, 0.15]
    net.set_master(m)
    return net


# eg1023 runs two warps per frame, eg4095 four
@pytest.mark.parametrize("key,p,F,ebn0", [("eg1023", 8, 300, 3.25), ("eg4095", 64, 96, 3.75)])
def test_decode_learned_replays_exactly(fwbf, key, p, F, ebn0):
    """The (alpha_q, theta_q) the network chose are recorded; the oracle run
    with that schedule reproduces every frame solved in the learned passes, and
    plain FWBF reproduces every frame handed to the fallback."""
    h, c, q = frames(key, F, ebn0, seed=44)
    k_learn, K = 6, 60
    net = _varied_network()
    with fwbf.Code.from_parity_check(h, p) as code:
        bits, iters = code.outputs(F)
        sched = torch.full((F, k_learn, 2), -1, dtype=torch.int32, device="cuda")
        fwbf.fwbf_decode_learned(code.handle, torch.from_numpy(q).cuda(), K, k_learn, 1.5, net.blob, bits, iters,
                                 out_sched=sched)
        torch.cuda.synchronize()
    it = iters.cpu().numpy()
    b = bits.cpu().numpy().view(np.uint32)
    s = sched.cpu().numpy()
    assert len(np.unique(s[:, 0, 0])) > 3  # the network really varies alpha
    learned = (it >= 0) & (it <= k_learn)
    A = np.full((F, K), 384, dtype=np.int32)
    T = np.zeros((F, K), dtype=np.int32)
    A[:, :k_learn] = np.where(s[:, :, 0] >= 0, s[:, :, 0], 384)
    T[:, :k_learn] = np.where(s[:, :, 1] >= 0, s[:, :, 1], 0)
    bo, io = oracle.fwbf_i8(h, p, q[learned], K, alpha_sched=A[learned], theta_sched=T[learned])
    assert np.array_equal(io, it[learned]) and np.array_equal(bo, b[learned])
    fb = ~learned
    bp, ip = oracle.fwbf_i8(h, p, q[fb], K, alpha=1.5)
    assert np.array_equal(bp, b[fb])
    assert np.array_equal(np.where(ip >= 0, ip + k_learn, ip), it[fb])


@pytest.mark.parametrize("key,p,F,ebn0", [("eg1023", 8, 120, 3.25), ("eg4095", 64, 48, 3.75)])
def test_learned_schedule_is_network_output(fwbf, key, p, F, ebn0):
    """Every (alpha_q, theta_q) a learned pass used is the network of the
    float64 oracle evaluated on that pass's recorded features: alpha_q =
    rne(256 clamp(o0, 0, 64)), theta_q = rne(256 clamp(16 o1, 0, 4096)).  The
    kernel computes in float32 (an error below 1e-5 per output for these
    weights), so each integer lies within half a unit of the exact value plus
    256 x 1e-5 (alpha_q) or 4096 x 1e-5 (theta_q)."""
    h, c, q = frames(key, F, ebn0, seed=45)
    k_learn, K = 6, 60
    net = _varied_network()
    with fwbf.Code.from_parity_check(h, p) as code:
        bits, iters = code.outputs(F)
        sched = torch.full((F, k_learn, 2), -1, dtype=torch.int32, device="cuda")
        feat = torch.full((F, k_learn, 8), np.nan, device="cuda")
        fwbf.fwbf_decode_learned(code.handle, torch.from_numpy(q).cuda(), K, k_learn, 1.5, net.blob, bits, iters,
                                 out_sched=sched, out_feat=feat)
        torch.cuda.synchronize()
    s = sched.cpu().numpy().reshape(-1, 2)
    x = feat.cpu().numpy().reshape(-1, 8)
    ran = s[:, 0] >= 0
    assert ran.sum() > F and not np.isnan(x[ran]).any()
    out, _ = mlp_ref.forward(net.master.cpu().numpy(), x[ran].astype(np.float64))
    aq = 256.0 * np.clip(out[:, 0], 0.0, 64.0)
    tq = 256.0 * np.clip(16.0 * out[:, 1], 0.0, 4096.0)
    assert np.abs(s[ran, 0] - aq).max() <= 0.5 + 256 * 1e-5
    assert np.abs(s[ran, 1] - tq).max() <= 0.5 + 4096 * 1e-5
    assert len(np.unique(s[ran, 0])) > 3 and len(np.unique(s[ran, 1])) > 3


def test_batched_learned_job_equals_single_code(fwbf):
    """A learned EG(4095) job (four warps per frame in the batch and alone), a
    learned EG(1023) job (one warp per frame in the batch, two alone) and a
    plain EG(1023) job give exactly the single-code results: the network's
    arithmetic order does not depend on how many warps evaluate it."""
    net = _varied_network()
    specs, singles, codes = [], [], []
    try:
        for key, p, F, learned in (("eg4095", 64, 150, True), ("eg1023", 16, 400, True),
                                   ("eg1023", 31, 400, False)):
            h, c, q = frames(key, F, 3.75, seed=45)
            code = fwbf.Code.from_parity_check(h, p)
            codes.append(code)
            qd = torch.from_numpy(q).cuda()
            b1, i1 = code.outputs(F)
            if learned:
                fwbf.fwbf_decode_learned(code.handle, qd, 60, 4, 1.5, net.blob, b1, i1)
            else:
                fwbf.fwbf_decode(code.handle, qd, 60, 1.5, b1, i1)
            b2, i2 = code.outputs(F)
            specs.append((code.handle, qd, 60, 1.5, b2, i2) + ((net.blob, 4) if learned else ()))
            singles.append((b1, i1, b2, i2))
        for packed in (1, 2):  # one warp per frame where 16 fit a block; warp groups everywhere
            for _, _, b2, i2 in singles:
                b2.fill_(-1)
                i2.fill_(-99)
            batch = fwbf.fwbf_batch_create(specs, warps_per_cta=16, packed=packed)
            try:
                fwbf.fwbf_decode_batch(batch)
                torch.cuda.synchronize()
                assert fwbf.fwbf_batch_status() == 0
            finally:
                fwbf.fwbf_batch_destroy(batch)
            for b1, i1, b2, i2 in singles:
                assert torch.equal(i1, i2) and torch.equal(b1, b2), packed
    finally:
        for code in codes:
            code.close()


def test_trained_network_gain(fwbf):
    """Train on frames plain FWBF labels itself, then compare on held-out
    frames: the learned schedule (with plain fallback) must not lose frames
    plain FWBF decodes, and must keep at most the plain frame error count."""
    from paper_1206_3362_gb300 import learned
    from paper_1206_3362_gb300.inputs import Encoder

    h = make_code("eg1023")
    enc = Encoder(h)
    sch = learned.Schedule(k_learn=6, label_max_iter=24)
    with fwbf.Code.from_parity_check(h, 8) as code:
        net, summary = learned.train_pipeline(code, enc, 1 << 15, (3.0, 3.5, 4.0), sch, epochs=3, seed=2,
                                              log=lambda *_: None)
        assert summary["losses"][-1] < summary["losses"][0]
        q, c = learned.make_frames(code, enc, 1 << 15, (3.25, 3.75), seed=99, device="cuda")
        plain = learned.evaluate(code, q, c, None, sch, reps=1)
        lrn = learned.evaluate(code, q, c, net, sch, reps=1)
    print("plain", plain, "learned", lrn, "train", summary)
    assert lrn["frame_errors"] <= plain["frame_errors"] + 3
