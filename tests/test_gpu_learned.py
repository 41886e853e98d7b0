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
    # the blob's order (include/fwbf.h): W1 and W3 as in the master vector, W2
    # (unit u, input c) at group 64 (c // 8) + u, element c % 8
    u, c = np.divmod(np.arange(4096), 64)
    order = np.concatenate([np.arange(512), 512 + 512 * (c // 8) + 8 * u + c % 8, np.arange(4608, 4736)])
    assert np.array_equal(w.view(np.float32)[order],
                          mlp_ref.bf16_round(dm.cpu().numpy()[:4736]).astype(np.float32))


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


def _default_network(alpha):
    """A network whose outputs are the fallback parameters for every input."""
    from paper_1206_3362_gb300.learned import Network

    net = Network(seed=9)
    m = net.master.cpu().numpy()
    m[4608:4736] = 0.0
    m[4864:4866] = [alpha, 0.0]
    net.set_master(m)
    return net


# eg1023 runs two warps per frame, eg4095 four
@pytest.mark.parametrize("key,p,F,ebn0", [("eg1023", 8, 300, 3.25), ("eg4095", 64, 96, 3.75)])
def test_decode_learned_replays_exactly(fwbf, key, p, F, ebn0):
    """The (alpha_q, theta_q) the network chose are recorded; the oracle run
    with that schedule reproduces every frame the learned passes solved, and
    every other frame carries plain FWBF's own result (the fallback).  The
    learned body that records nothing gives the same results."""
    h, c, q = frames(key, F, ebn0, seed=44)
    k_learn, K = 6, 60
    net = _varied_network()
    with fwbf.Code.from_parity_check(h, p) as code:
        bits, iters = code.outputs(F)
        sched = torch.full((F, k_learn, 2), -1, dtype=torch.int32, device="cuda")
        qd = torch.from_numpy(q).cuda()
        fwbf.fwbf_decode_learned(code.handle, qd, K, k_learn, 1.5, net.blob, bits, iters, out_sched=sched)
        b2, i2 = code.outputs(F)
        fwbf.fwbf_decode_learned(code.handle, qd, K, k_learn, 1.5, net.blob, b2, i2)
        torch.cuda.synchronize()
    assert torch.equal(iters, i2) and torch.equal(bits, b2)
    it = iters.cpu().numpy()
    b = bits.cpu().numpy().view(np.uint32)
    s = sched.cpu().numpy()
    used = s[s[:, :, 0] >= 0]  # (alpha_q, theta_q) of every learned pass that ran
    # the network really varies both parameters, and some passes keep plain FWBF's
    assert len(np.unique(used[:, 0])) >= 3 and len(np.unique(used[:, 1])) >= 2
    assert ((used[:, 0] == 384) & (used[:, 1] == 0)).any()
    A = np.full((F, K), 384, dtype=np.int32)
    T = np.zeros((F, K), dtype=np.int32)
    A[:, :k_learn] = np.where(s[:, :, 0] >= 0, s[:, :, 0], 384)
    T[:, :k_learn] = np.where(s[:, :, 1] >= 0, s[:, :, 1], 0)
    bo, io = oracle.fwbf_i8(h, p, q, K, alpha_sched=A, theta_sched=T)
    learned = (io >= 0) & (io <= k_learn)  # solved within the learned passes
    assert learned.sum() >= 8 and (~learned).sum() >= 8
    assert np.array_equal(io[learned], it[learned]) and np.array_equal(bo[learned], b[learned])
    fb = ~learned
    bp, ip = oracle.fwbf_i8(h, p, q[fb], K, alpha=1.5)
    assert np.array_equal(bp, b[fb]) and np.array_equal(ip, it[fb])


@pytest.mark.parametrize("key,p,F,ebn0", [("eg1023", 8, 400, 3.0), ("eg4095", 64, 96, 3.75)])
def test_learned_default_network_is_plain(fwbf, key, p, F, ebn0):
    """A network that always answers the fallback parameters (alpha 1.5,
    threshold 0) decodes every frame exactly as plain FWBF does: no pass
    deviates, so frames still unsolved after k_learn passes continue from
    plain FWBF's own state, and a gated pass without flips is plain FWBF's
    fixed point."""
    h, c, q = frames(key, F, ebn0, seed=46)
    net = _default_network(1.5)
    with fwbf.Code.from_parity_check(h, p) as code:
        bits, iters = code.outputs(F)
        fwbf.fwbf_decode_learned(code.handle, torch.from_numpy(q).cuda(), 60, 3, 1.5, net.blob, bits, iters)
        torch.cuda.synchronize()
    it = iters.cpu().numpy()
    bp, ip = oracle.fwbf_i8(h, p, q, 60, alpha=1.5)
    assert (it > 3).sum() > 0 and (it < 0).sum() > 0  # continued frames and failures are both covered
    assert np.array_equal(ip, it) and np.array_equal(bp, bits.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("key,p,F,ebn0", [("eg1023", 8, 120, 3.25), ("eg4095", 64, 48, 3.75)])
def test_learned_schedule_is_network_output(fwbf, key, p, F, ebn0):
    """Every (alpha_q, theta_q) a learned pass used is the network of the
    float64 oracle evaluated on that pass's recorded features, snapped to the
    grid: alpha_q = 128 rne(2 clamp(o0, 0, 64)), theta_q = 1024 rne(clamp(4 o1,
    0, 1024)).  The kernel computes in float32 (an error below 1e-5 per output
    for these weights), so where the exact value lies within 1e-4 of a
    rounding boundary either neighbour is accepted.  Passes with a syndrome
    weight below 6 d_v use the fallback parameters (alpha_q 384, theta_q 0)."""
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
    dv = int(np.max(h.col_weights()))
    W = np.rint(x[:, 0].astype(np.float64) * h.N)
    gated = (s[:, 0] >= 0) & (W < 6 * dv)
    assert gated.any()
    assert (s[gated, 0] == 384).all() and (s[gated, 1] == 0).all()
    ran = (s[:, 0] >= 0) & ~gated
    assert ran.sum() > F and not np.isnan(x[ran]).any()
    out, _ = mlp_ref.forward(net.master.cpu().numpy(), x[ran].astype(np.float64))

    def snapped_ok(got, v, unit):
        # got / unit must be rne(v), or either neighbour of a near-tie
        lo, hi = np.floor(v), np.ceil(v)
        near_tie = np.abs(v - np.floor(v) - 0.5) < 1e-4
        want = np.round(v)  # round half to even, as the kernel's rne
        k = got / unit
        return (k == want) | (near_tie & ((k == lo) | (k == hi)))

    assert (s[ran] % [128, 1024] == 0).all()
    assert snapped_ok(s[ran, 0], 2.0 * np.clip(out[:, 0], 0.0, 64.0), 128).all()
    assert snapped_ok(s[ran, 1], np.clip(4.0 * out[:, 1], 0.0, 1024.0), 1024).all()
    assert len(np.unique(s[ran, 0])) >= 3 and len(np.unique(s[ran, 1])) >= 2


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
    """What the committed EG(1023,781) network gains over the method without
    it, on 2^18 held-out seeded frames at 4 dB: plain FWBF with the same block
    length and weighting factor (the learned decoder's own fallback) against
    the learned schedule.  The learned frame error rate's 95 % Wilson interval
    lies entirely below plain FWBF's, and no frame that plain FWBF decodes to
    the transmitted codeword is lost."""
    from paper_1206_3362_gb300 import learned
    from paper_1206_3362_gb300.inputs import Encoder

    h = make_code("eg1023")
    enc = Encoder(h)
    net = learned.Network()
    meta = net.load(learned.DEFAULT_WEIGHTS)
    p, alpha, k_learn = int(meta["seg_len"]), float(meta["alpha_default"]), int(meta["k_learn"])
    with fwbf.Code.from_parity_check(h, p) as code:
        q, c = learned.make_frames(code, enc, 1 << 18, (4.0,), seed=4242, device="cuda")
        bp, ip = code.outputs(q.shape[0])
        fwbf.fwbf_decode(code.handle, q, 100, alpha, bp, ip)
        bl, il = code.outputs(q.shape[0])
        fwbf.fwbf_decode_learned(code.handle, q, 100, k_learn, alpha, net.blob, bl, il)
        torch.cuda.synchronize()
    ok_plain = learned.frame_ok(bp, ip, c)
    ok_learned = learned.frame_ok(bl, il, c)
    n = q.shape[0]
    fe_plain, fe_learned = int((~ok_plain).sum()), int((~ok_learned).sum())
    lo_plain, _ = learned.wilson(fe_plain, n)
    _, hi_learned = learned.wilson(fe_learned, n)
    print(f"frame errors: plain {fe_plain}, learned {fe_learned} of {n}")
    assert hi_learned < lo_plain
    assert int((ok_plain & ~ok_learned).sum()) == 0


def test_train_pipeline_smoke(fwbf):
    """Labels, features and training from scratch on 2^15 frames (a quick run
    of the whole pipeline): the loss falls, and on held-out frames the new
    network keeps at most the plain frame error count plus a small margin."""
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
    assert lrn["frame_errors"] <= plain["frame_errors"] * 1.1 + 5
