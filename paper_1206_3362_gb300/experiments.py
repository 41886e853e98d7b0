"""Simulation experiments of the paper's Sec. V, run with the GPU decoders.

* ``tab1``: averaged iterations on EG(1023,781) with K_max = 10 (Tab. 1) for
  FWBF with p = 31 and p = 93, for lambda-largest selection (MLP-WBF's
  bit-choose rule, lambda = 10, here with the IMWBF metric since the paper
  does not define the LP metric), and for single-bit IMWBF flipping (p = N).
  Iterations are counted as the paper's table appears to: evaluations of Step 1
  (flip passes + 1; K_max + 1 for a frame that does not converge).
* ``eg255``: FWBF BER / FER of the EG(255,175) code (the paper's code 1) over
  Eb/N0 for two block lengths and K_max = 5 and 10 (the paper notes that 5 and 10
  iterations are not distinctly apart).

* ``sweep1``: plain FWBF on EG(1023,781) over 3.0-5.0 dB in 0.25 dB steps
  (FER, BER, passes, throughput per point).
* ``scale4``: learned + batched at scale: the rate-0.94 quasi-cyclic N = 16384
  code (column weight 4, circulants of 512) and EG(4095,3367), 2^22 frames over
  4.0-5.5 dB, one graph-captured batched launch with autotuned block lengths
  and the learned schedule on the EG code, against plain FWBF (paper setting,
  one launch per code and point) on the same frames.  Frames reuse a pool of
  seeded codewords under fresh seeded noise (FWBF's outcome depends only on the
  error pattern and |y|, not on which codeword was sent).
* ``kernels``: one launch of each benchmarked decode kernel on 131,072
  EG(1023,781) frames at 4 dB (134 MB of int8 frames, more than L2): plain
  FWBF in the paper setting (p = 31, alpha = 1.5) and the learned + batched
  form (p = 8, alpha 2, gate 14 d_v); a small case for profilers.
* ``qc``: plain FWBF (paper setting) on the quasi-cyclic N = 16384 and
  N = 8192 codes at 4 dB: the packed quasi-cyclic decoder, and the list decoder
  on the same code with its checks (rows) permuted -- no circulant structure
  left, but the same metric for every bit, so the same results on the same
  frames.  (Permuting bits would not do: the p-bit blocks follow bit order.)

    python -m paper_1206_3362_gb300.experiments tab1 [--frames N]
    python -m paper_1206_3362_gb300.experiments eg255 [--frames N]
    python -m paper_1206_3362_gb300.experiments scale4 [--frames N]
    python -m paper_1206_3362_gb300.experiments sweep1 [--frames N]
    python -m paper_1206_3362_gb300.experiments qc [--frames N]
    python -m paper_1206_3362_gb300.experiments kernels [--frames N]
"""
from __future__ import annotations

import json
import os

from . import fwbf
from .learned import frame_ok, make_frames, unpack_bits_torch, wilson

TAB1 = {"ebn0_db": (3.0, 3.5, 4.0, 4.5), "mlp_wbf": (8.86, 6.20, 4.54, 3.83),
        "fwbf_p93": (9.29, 7.37, 6.06, 5.12), "fwbf_p31": (8.62, 5.60, 4.19, 3.64)}


def _run(code, q, c, max_iter, alpha, lam=None):
    import torch

    bits, iters = code.outputs(q.shape[0], q.device)
    if lam is None:
        fwbf.fwbf_decode(code.handle, q, max_iter, alpha, bits, iters)
    else:
        fwbf.fwbf_decode_lambda(code.handle, q, max_iter, alpha, lam, bits, iters)
    torch.cuda.synchronize()
    ok = frame_ok(bits, iters, c)
    steps = torch.where(iters >= 0, iters + 1, torch.full_like(iters, max_iter + 1)).float().mean().item()
    fe = int((~ok).sum().item())
    be = int((unpack_bits_torch(bits, c.shape[1]) != c).sum().item())
    return {"avg_step1": steps, "fer": fe / q.shape[0], "fer_ci95": wilson(fe, q.shape[0]),
            "ber": be / (q.shape[0] * c.shape[1])}


def tab1(frames: int = 1 << 16, alpha: float = 1.5):
    from .inputs import Encoder, make_code

    h = make_code("eg1023")
    enc = Encoder(h)
    codes = {p: fwbf.Code.from_parity_check(h, p) for p in (31, 93, h.N)}
    out = {"paper_tab1": TAB1, "frames": frames, "alpha": alpha, "rows": {}}
    for i, eb in enumerate(TAB1["ebn0_db"]):
        q, c = make_frames(codes[31], enc, frames, (eb,), seed=900 + i, device="cuda")
        row = {"fwbf_p31": _run(codes[31], q, c, 10, alpha), "fwbf_p93": _run(codes[93], q, c, 10, alpha),
               "lambda10_imwbf": _run(codes[31], q, c, 10, alpha, lam=10),
               "imwbf_single_flip": _run(codes[h.N], q, c, 10, alpha)}
        out["rows"][f"{eb}dB"] = row
    for code in codes.values():
        code.close()
    return out


def eg255(frames: int = 1 << 17, alpha: float = 1.5, ebn0=(3.0, 3.5, 4.0, 4.5, 5.0, 5.5, 6.0)):
    from .inputs import Encoder, make_code

    h = make_code("eg255")
    enc = Encoder(h)
    codes = {p: fwbf.Code.from_parity_check(h, p) for p in (16, 51)}
    out = {"frames": frames, "alpha": alpha, "rows": {}}
    for i, eb in enumerate(ebn0):
        q, c = make_frames(codes[16], enc, frames, (eb,), seed=700 + i, device="cuda")
        out["rows"][f"{eb}dB"] = {f"p{p}_kmax{k}": _run(codes[p], q, c, k, alpha) for p in (16, 51) for k in (5, 10)}
    for code in codes.values():
        code.close()
    return out


def sweep1(frames: int = 1 << 20, p: int = 31, alpha: float = 1.5, max_iter: int = 100,
           ebn0=tuple(3.0 + 0.25 * i for i in range(9))):
    """Plain FWBF on EG(1023,781) over 3.0-5.0 dB: FER (Wilson 95 % interval),
    BER over the information bits and over all N bits, converged passes,
    decode time and decoded information Gb/s per point."""
    import torch

    from .inputs import Encoder, make_code

    h = make_code("eg1023")
    enc = Encoder(h)
    info = torch.as_tensor(enc.info_pos, device="cuda")
    out = {"code": "eg1023", "p": p, "alpha": alpha, "max_iter": max_iter, "frames": frames, "rows": {}}
    with fwbf.Code.from_parity_check(h, p) as code:
        for i, eb in enumerate(ebn0):
            q, c = make_frames(code, enc, frames, (eb,), seed=1100 + i, device="cuda")
            bits, iters = code.outputs(frames, q.device)
            fwbf.fwbf_decode(code.handle, q, max_iter, alpha, bits, iters)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fwbf.fwbf_decode(code.handle, q, max_iter, alpha, bits, iters)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            ok = frame_ok(bits, iters, c)
            fe = int((~ok).sum().item())
            wrong = unpack_bits_torch(bits, h.N) != c
            conv = iters >= 0
            out["rows"][f"{eb}dB"] = {
                "fer": fe / frames, "fer_ci95": wilson(fe, frames),
                "ber_info": float(wrong[:, info].float().mean().item()),
                "ber_all": float(wrong.float().mean().item()),
                "avg_passes_converged": float(iters[conv].float().mean().item()) if conv.any() else None,
                "decode_ms": ms, "gbps": frames * enc.K / ms / 1e6}
            del q, c, bits, iters, wrong
    return out


SCALE4_CODES = (("qc16384", 32), ("eg4095", 64))  # (code, the paper-setting block length p)
SCALE4_EBN0 = (4.0, 4.5, 5.0, 5.5)


def _pool_frames(enc, pool_c, n, ebn0, seed, device, chunk=1 << 15):
    """n quantised frames: codeword pool_c[i mod P] plus fresh seeded AWGN."""
    import torch

    from .inputs.channel import awgn_sigma

    P, N = pool_c.shape
    q = torch.empty((n, N), dtype=torch.int8, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + int(round(ebn0 * 1000)))
    sigma = awgn_sigma(ebn0, enc.rate)
    for s0 in range(0, n, chunk):
        m = min(chunk, n - s0)
        idx = torch.arange(s0, s0 + m, device=device) % P
        y = (1.0 - 2.0 * pool_c[idx].to(torch.float32)) + sigma * torch.randn((m, N), generator=g, device=device)
        fwbf.fwbf_quantize(y.contiguous(), q[s0:s0 + m])
    return q


def _errors(bits, iters, pool_c, chunk=1 << 15):
    import torch

    from .learned import unpack_bits_torch

    P, N = pool_c.shape
    fe = be = 0
    for s0 in range(0, bits.shape[0], chunk):
        b = bits[s0:s0 + chunk]
        idx = torch.arange(s0, s0 + b.shape[0], device=bits.device) % P
        wrong = unpack_bits_torch(b, N) != pool_c[idx]
        fe += int((wrong.any(dim=1) | (iters[s0:s0 + chunk] < 0)).sum().item())
        be += int(wrong.sum().item())
    return fe, be


def scale4(frames: int = 1 << 22, reps: int = 2, weights: dict | None = None, max_iter: int = 100, clocks=None):
    import time

    import torch

    from . import autotune
    from .inputs import Encoder, make_code
    from .inputs.channel import random_codewords_torch
    from .learned import Network, weights_path

    dev = "cuda"
    per_job = frames // (len(SCALE4_CODES) * len(SCALE4_EBN0))
    jobs, handles = [], []
    out = {"frames": per_job * len(SCALE4_CODES) * len(SCALE4_EBN0), "frames_per_job": per_job,
           "ebn0_db": SCALE4_EBN0, "max_iter": max_iter, "codes": {}, "jobs": []}
    t0 = time.time()
    for ci, (key, p_ref) in enumerate(SCALE4_CODES):
        h = make_code(key)
        enc = Encoder(h)
        pool = 1 << 13 if h.N > 8192 else 1 << 14
        _, pool_c = random_codewords_torch(enc, pool, seed=4000 + ci, device=dev)
        tune = autotune.tune_code(h, enc, SCALE4_EBN0[1], p_ref=p_ref, alpha_ref=1.5, frames=1 << 14)
        p_t, a_t = tune["choice"]["p"], tune["choice"]["alpha"]
        net, k_learn, gate = None, 0, None
        wpath = (weights or {}).get(key, weights_path(key))
        if os.path.exists(wpath):
            net = Network(alpha_default=a_t)
            meta = net.load(wpath)
            p_t, a_t, k_learn = int(meta["seg_len"]), float(meta["alpha_default"]), int(meta["k_learn"])
        code_ref = fwbf.Code.from_parity_check(h, p_ref)
        code_t = fwbf.Code.from_parity_check(h, p_t)
        handles += [code_ref, code_t]
        if net is not None:  # the gate of the learned schedule, on calibration frames at the lowest point
            qcal = _pool_frames(enc, pool_c, 1 << 16, SCALE4_EBN0[0], seed=6000 + ci, device=dev)
            ccal = pool_c[torch.arange(1 << 16, device=dev) % pool_c.shape[0]]
            gate = autotune.tune_gate(code_t, qcal, ccal, net, a_t, k_learn, max_iter=max_iter, reps=2)
            del qcal, ccal
        out["codes"][key] = {"N": h.N, "K": enc.K, "rate": enc.rate, "p_paper": p_ref, "p_tuned": p_t,
                             "alpha_tuned": a_t, "learned": net is not None, "k_learn": k_learn,
                             "gate_dv": gate["choice"] if gate else None, "gate_tuning": gate,
                             "codeword_pool": pool, "autotune": tune["choice"]}
        for pi, eb in enumerate(SCALE4_EBN0):
            q = _pool_frames(enc, pool_c, per_job, eb, seed=5000 + 10 * ci + pi, device=dev)
            jobs.append(dict(key=key, ebn0=eb, K=enc.K, q=q, pool_c=pool_c, code_ref=code_ref, code_t=code_t,
                             a_t=a_t, net=net, k_learn=k_learn, gate_dv=gate["choice"] if gate else 0,
                             plain=code_ref.outputs(per_job, dev),
                             batched=code_t.outputs(per_job, dev)))
    torch.cuda.synchronize()
    out["generate_seconds"] = time.time() - t0
    info_bits = sum(j["K"] * per_job for j in jobs)

    # plain FWBF, paper setting: one launch per code and point
    def plain():
        for j in jobs:
            fwbf.fwbf_decode(j["code_ref"].handle, j["q"], max_iter, 1.5, *j["plain"])

    plain()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.mark("plain")
    e0.record()
    for _ in range(reps):
        plain()
    e1.record()
    torch.cuda.synchronize()
    if clocks:
        clocks.unmark("plain")
    ms_plain = e0.elapsed_time(e1) / reps

    # learned + batched: one graph-captured launch over every code and point
    spec = []
    for j in jobs:
        job = (j["code_t"].handle, j["q"], max_iter, j["a_t"], *j["batched"])
        if j["net"] is not None:
            job = job + (j["net"].blob, j["k_learn"], j["gate_dv"])
        spec.append(job)
    # CTA shape tuned on 1/16 of every job's frames (the packed decoder with and
    # without warp groups; the list decoder gives the same results, slower)
    sub = max(1, per_job // 16)
    small = [(j[0], j[1][:sub], j[2], j[3], j[4][:sub], j[5][:sub]) + tuple(j[6:]) for j in spec]
    shape, _ = autotune.tune_batch_shape(small, warps_candidates=(8, 16), packed_candidates=(2, 1))
    batch = fwbf.fwbf_batch_create(spec, warps_per_cta=shape["warps_per_cta"], packed=shape["packed"])
    s = torch.cuda.Stream()
    try:
        with torch.cuda.stream(s):
            fwbf.fwbf_decode_batch(batch, s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            fwbf.fwbf_decode_batch(batch, s)
        with torch.cuda.stream(s):
            g.replay()
            torch.cuda.synchronize()
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if clocks:
                clocks.mark("learned_batched")
            b0.record(s)
            for _ in range(reps):
                g.replay()
            b1.record(s)
        torch.cuda.synchronize()
        if clocks:
            clocks.unmark("learned_batched")
        assert fwbf.fwbf_batch_status() == 0
        ms_batched = b0.elapsed_time(b1) / reps
    finally:
        fwbf.fwbf_batch_destroy(batch)

    for j in jobs:
        row = {"code": j["key"], "ebn0_db": j["ebn0"], "frames": per_job}
        for arm in ("plain", "batched"):
            bits, iters = j[arm]
            fe, be = _errors(bits, iters, j["pool_c"])
            row[arm] = {"fer": fe / per_job, "fer_ci95": wilson(fe, per_job),
                        "ber": be / (per_job * j["pool_c"].shape[1]),
                        "failed_frac": float((iters < 0).float().mean().item())}
        out["jobs"].append(row)
    out["plain"] = {"ms": ms_plain, "gbps": info_bits / (ms_plain / 1e3) / 1e9, "launches": len(jobs)}
    out["learned_batched"] = {"ms": ms_batched, "gbps": info_bits / (ms_batched / 1e3) / 1e9, "launches": 1,
                              "shape": shape}
    for code in handles:
        code.close()
    return out


QC_CODES = (("qc16384", 32), ("qc8192", 64))  # (code, block length p)


def qc_decoders(frames: int = 1 << 16, reps: int = 3, ebn0: float = 4.0, max_iter: int = 100,
                alpha: float = 1.5):
    import numpy as np
    import torch

    from .inputs import Encoder, make_code
    from .inputs.channel import random_codewords_torch
    from .inputs.codes import ParityCheck

    out = {"frames": frames, "ebn0_db": ebn0, "max_iter": max_iter, "alpha": alpha, "codes": {}}
    for ci, (key, p) in enumerate(QC_CODES):
        h = make_code(key)
        enc = Encoder(h)
        _, pool_c = random_codewords_torch(enc, 1 << 13, seed=6000 + ci, device="cuda")
        q = _pool_frames(enc, pool_c, frames, ebn0, seed=6100 + ci, device="cuda")
        perm = np.random.default_rng(ci).permutation(h.M)
        hp = ParityCheck(N=h.N, M=h.M, rows=perm[h.rows].astype(np.int32), cols=h.cols)
        row = {"N": h.N, "K": enc.K, "p": p}
        res = {}
        for name, hh, qq in (("packed_qc", h, q), ("list", hp, q)):
            with fwbf.Code.from_parity_check(hh, p) as code:
                bits, iters = code.outputs(frames)
                fwbf.fwbf_decode(code.handle, qq, max_iter, alpha, bits, iters)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    fwbf.fwbf_decode(code.handle, qq, max_iter, alpha, bits, iters)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                res[name] = (bits, iters)
                row[name] = {"decoder": int(code.info.decoder), "ms": ms,
                             "gbps": frames * enc.K / (ms / 1e3) / 1e9,
                             "failed_frac": float((iters < 0).float().mean().item())}
        (b0, i0), (b1, i1) = res["packed_qc"], res["list"]
        row["identical"] = bool(torch.equal(i0, i1)) and bool(torch.equal(b0, b1))
        row["speedup"] = row["list"]["ms"] / row["packed_qc"]["ms"]
        out["codes"][key] = row
    return out


def kernels(frames: int = 1 << 17, gate_dv: int = 14):
    """One plain FWBF decode (p = 31, alpha = 1.5) and one graph-free
    learned + batched launch (the committed network, its p and alpha, gate
    gate_dv) of the same seeded frames; returns their failure counts."""
    import torch

    from .inputs import Encoder, make_code
    from .inputs.channel import bpsk_awgn_torch, random_codewords_torch
    from .learned import DEFAULT_WEIGHTS, Network

    h = make_code("eg1023")
    enc = Encoder(h)
    _, c = random_codewords_torch(enc, frames, seed=7, device="cuda")
    q = fwbf.quantize(bpsk_awgn_torch(c, 4.0, enc.rate, seed=7).contiguous())
    net = Network(alpha_default=2.0)
    meta = net.load(DEFAULT_WEIGHTS)
    p_l, a_l, k_l = int(meta["seg_len"]), float(meta["alpha_default"]), int(meta["k_learn"])
    with fwbf.Code.from_parity_check(h, 31) as code31, fwbf.Code.from_parity_check(h, p_l) as code_l:
        b31, i31 = code31.outputs(frames)
        fwbf.fwbf_decode(code31.handle, q, 100, 1.5, b31, i31)
        bl, il = code_l.outputs(frames)
        batch = fwbf.fwbf_batch_create([(code_l.handle, q, 100, a_l, bl, il, net.blob, k_l, gate_dv)],
                                       warps_per_cta=16, packed=2)
        try:
            fwbf.fwbf_decode_batch(batch)
            torch.cuda.synchronize()
        finally:
            fwbf.fwbf_batch_destroy(batch)
        return {"frames": frames, "plain_failed": int((i31 < 0).sum()), "learned_failed": int((il < 0).sum())}


def main():
    import argparse

    import torch

    import __graft_entry__

    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["tab1", "eg255", "scale4", "sweep1", "qc", "kernels"])
    ap.add_argument("--frames", type=int, default=None)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    __graft_entry__.build()
    torch.cuda.set_device(0)
    if args.what == "tab1":
        res = tab1(args.frames or (1 << 16))
    elif args.what == "eg255":
        res = eg255(args.frames or (1 << 17))
    elif args.what == "sweep1":
        res = sweep1(args.frames or (1 << 20))
    elif args.what == "qc":
        res = qc_decoders(args.frames or (1 << 16))
    elif args.what == "kernels":
        res = kernels(args.frames or (1 << 17))
    else:
        res = scale4(args.frames or (1 << 22))
    text = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
