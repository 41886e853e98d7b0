"""Autotuner for the decoder's free parameters on the running GPU.

Tuned per code, on seeded calibration frames at a chosen Eb/N0:

* block length p of the partially parallel bit-choose and the weighting factor
  alpha -- both change results, so a candidate is admitted only if it is
  FER-qualified: on the same calibration frames it has at most the frame
  errors and at most the bit errors of the reference setting (the paper's p
  and alpha; the bit errors decide on codes where every setting fails every
  frame);
* the decoder variant ("bit-packing width": the packed cyclic decoder with two
  positions per 32-bit register, or the list decoder with one), and, for a
  batch, the number of warps per CTA and whether every frame is decoded by a
  group of warps ("lanes per frame": packed = 2).

* the gate of the learned schedule (the network is consulted on passes with
  W_k >= gate_dv d_v): a gate is admitted if it keeps at least half of the
  network's frame-error gain, i.e. its frame errors are at most the midpoint
  between those of the network consulted on every pass and those of plain
  FWBF with the same p and alpha (select_gate).

Among admitted settings the fastest (CUDA-event time of the decode) wins.
Results are cached in a JSON file keyed by code, Eb/N0 and GPU name.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import fwbf

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "fwbf", "autotune.json")
P_CANDIDATES = (1, 2, 4, 8, 16, 32, 64)
ALPHA_CANDIDATES = (1.0, 1.5, 2.0, 2.5)


def code_key(h) -> str:
    d = hashlib.sha1()
    d.update(np.asarray([h.N, h.M], dtype=np.int64).tobytes())
    d.update(np.asarray(h.rows, dtype=np.int32).tobytes())
    d.update(np.asarray(h.cols, dtype=np.int32).tobytes())
    return d.hexdigest()[:16]


def _time(fn, reps=3):
    import torch

    fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def calibration_frames(h, enc, F, ebn0, seed, device="cuda"):
    from .inputs.channel import bpsk_awgn_torch, random_codewords_torch

    _, c = random_codewords_torch(enc, F, seed=seed, device=device)
    y = bpsk_awgn_torch(c, ebn0, enc.rate, seed=seed).contiguous()
    return fwbf.quantize(y), c


def _errors(bits, iters, c):
    """(frame errors, bit errors) against the transmitted codewords."""
    from .learned import frame_ok, unpack_bits_torch

    fe = int((~frame_ok(bits, iters, c)).sum().item())
    be = int((unpack_bits_torch(bits, c.shape[1]) != c).sum().item())
    return fe, be


def tune_code(h, enc, ebn0: float, p_ref: int, alpha_ref: float = 1.5, frames: int = 1 << 15,
              max_iter: int = 100, p_candidates=P_CANDIDATES, alpha_candidates=ALPHA_CANDIDATES,
              seed: int = 4242, log=None):
    """Fastest (p, alpha) for one code among the candidates with no more frame
    errors and no more bit errors than the reference (p_ref, alpha_ref) on the
    same seeded frames (bit errors decide between settings that all fail, as on
    codes beyond bit flipping's reach); returns a dict with the choice, the
    reference and every candidate measured."""
    q, c = calibration_frames(h, enc, frames, ebn0, seed)
    results = []
    ref = None
    cands = sorted({(p_ref, alpha_ref)} | {(p, a) for p in p_candidates if p <= h.N for a in alpha_candidates})
    for p, a in cands:
        with fwbf.Code.from_parity_check(h, p) as code:
            bits, iters = code.outputs(frames)
            ms = _time(lambda: fwbf.fwbf_decode(code.handle, q, max_iter, a, bits, iters))
            fe, be = _errors(bits, iters, c)
        r = {"p": p, "alpha": a, "frame_errors": fe, "bit_errors": be, "ms": ms}
        results.append(r)
        if (p, a) == (p_ref, alpha_ref):
            ref = r
        if log:
            log(r)
    best = select_fastest_qualified(results, ref)
    return {"choice": {"p": best["p"], "alpha": best["alpha"]}, "reference": ref, "candidates": results,
            "frames": frames, "ebn0_db": ebn0}


def select_fastest_qualified(results, ref):
    """The fastest of the measured settings whose frame errors and bit errors
    are both at most the reference's (the reference itself always qualifies);
    ties in time keep the earlier entry."""
    qualified = [r for r in results
                 if r["frame_errors"] <= ref["frame_errors"] and r["bit_errors"] <= ref["bit_errors"]]
    return min(qualified, key=lambda r: r["ms"])


GATE_CANDIDATES = (0, 6, 10, 12, 14, 16)


GATE_TIME_TIE = 0.01  # gates within 1 % of the fastest qualifying one count as equally fast


def select_gate(results, plain):
    """The fastest gate whose frame errors are at most the midpoint between
    the ungated network's (gate_dv = 0, which must be measured) and plain
    FWBF's; the ungated network always qualifies.  Qualifying gates within
    GATE_TIME_TIE of the fastest one's time are a tie (their differences are
    below the timing's run-to-run spread), decided by fewer frame errors, then
    fewer bit errors, then time, then the earlier entry."""
    full = next(r for r in results if r["gate_dv"] == 0)
    limit = (full["frame_errors"] + plain["frame_errors"]) / 2.0
    qualified = [r for r in results if r is full or r["frame_errors"] <= limit]
    fastest = min(r["ms"] for r in qualified)
    near = [r for r in qualified if r["ms"] <= fastest * (1.0 + GATE_TIME_TIE)]
    return min(near, key=lambda r: (r["frame_errors"], r["bit_errors"], r["ms"]))


def tune_gate(code, q, c, net, alpha: float, k_learn: int, max_iter: int = 100, candidates=GATE_CANDIDATES,
              reps: int = 3, log=None):
    """Measures the learned decoder (network blob net.blob) at every gate
    candidate and plain FWBF on the same calibration frames (q int8, c the
    transmitted codewords) and picks the gate by select_gate."""
    F = q.shape[0]
    bits, iters = code.outputs(F)
    ms = _time(lambda: fwbf.fwbf_decode(code.handle, q, max_iter, alpha, bits, iters), reps)
    fe, be = _errors(bits, iters, c)
    plain = {"frame_errors": fe, "bit_errors": be, "ms": ms}
    results = []
    for g in sorted(set(candidates) | {0}):
        ms = _time(lambda: fwbf.fwbf_decode_learned(code.handle, q, max_iter, k_learn, alpha, net.blob, bits, iters,
                                                    gate_dv=g), reps)
        fe, be = _errors(bits, iters, c)
        results.append({"gate_dv": g, "frame_errors": fe, "bit_errors": be, "ms": ms})
        if log:
            log(results[-1])
    best = select_gate(results, plain)
    return {"choice": best["gate_dv"], "plain": plain, "candidates": results, "frames": F}


def tune_batch_shape(jobs, warps_candidates=(4, 8, 12, 16), packed_candidates=(2, 1, 0)):
    """Fastest (warps_per_cta, packed) for a batch of jobs [(code, y, max_iter,
    alpha, bits, iters)]; every variant gives identical results.  packed = 2
    (warp groups, fixed 512-thread CTAs) is timed once, at 16 warps."""
    best = None
    rows = []
    for packed in packed_candidates:
        for w in ((16,) if packed == 2 else warps_candidates):
            b = fwbf.fwbf_batch_create(jobs, warps_per_cta=w, packed=packed)
            try:
                ms = _time(lambda: fwbf.fwbf_decode_batch(b))
            finally:
                fwbf.fwbf_batch_destroy(b)
            rows.append({"warps_per_cta": w, "packed": packed, "ms": ms})
            if best is None or ms < best["ms"]:
                best = rows[-1]
    return best, rows


class Cache:
    def __init__(self, path: str = DEFAULT_CACHE):
        self.path = path
        try:
            with open(path) as f:
                self.data = json.load(f)
        except (OSError, ValueError):
            self.data = {}

    def key(self, h, ebn0, what="code"):
        import torch

        return f"{what}:v2:{code_key(h)}:{ebn0:.3f}:{torch.cuda.get_device_name()}"  # v2: frame + bit errors

    def get(self, k):
        return self.data.get(k)

    def put(self, k, v):
        self.data[k] = v
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1)
        os.replace(tmp, self.path)


def tuned_code(h, enc, ebn0, p_ref, alpha_ref=1.5, cache: Cache | None = None, **kw):
    cache = cache or Cache()
    k = cache.key(h, ebn0)
    hit = cache.get(k)
    if hit is None:
        t0 = time.time()
        hit = tune_code(h, enc, ebn0, p_ref, alpha_ref, **kw)
        hit["tune_seconds"] = time.time() - t0
        cache.put(k, hit)
    return hit
