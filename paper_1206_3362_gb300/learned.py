"""Learned per-pass schedule for FWBF: labels, features, training, evaluation.

The paper's method has two parameters per pass: the weighting factor alpha of
Eq. 1 and the flip threshold of Sec. III Step 2 (0 in the paper).  A small
network (8 -> 64 -> 64 -> 2, BF16 weights, FP32 arithmetic) predicts both from
per-frame syndrome-weight and metric statistics (the features documented in
include/fwbf.h).  Everything runs on the GPU through the C ABI:

* labels: for every training frame and pass k, plain FWBF itself searches a
  small (alpha, theta) grid: the pass-k choice is the grid point after which
  plain FWBF (default parameters) reaches the transmitted codeword in the
  fewest passes, given the labels of the earlier passes (ties keep the
  default) -- fwbf_decode_sched;
* features along the labelled trajectories -- fwbf_decode_sched(out_feat);
* training: mean squared error on (alpha, theta / 16) with Adam --
  fwbf_mlp_grad / fwbf_mlp_adam (hand-written kernels);
* decoding: fwbf_decode_learned, with plain FWBF as the fallback for frames
  still unsolved after k_learn learned passes.
"""
from __future__ import annotations

import dataclasses
import math
import os
import time

import numpy as np

from . import fwbf

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
DEFAULT_WEIGHTS = os.path.join(WEIGHTS_DIR, "fwbf_mlp_eg1023.npz")


def weights_path(code_key: str) -> str:
    return os.path.join(WEIGHTS_DIR, f"fwbf_mlp_{code_key}.npz")


@dataclasses.dataclass
class Schedule:
    alpha_default: float = 1.5
    grid_alpha: tuple = (1.0, 1.5, 2.0, 2.5, 3.0)
    grid_theta: tuple = (0.0, 4.0, 8.0)   # in units of the int8 metric
    k_learn: int = 8
    gate_dv: int = 6          # the network is consulted on passes with W_k >= gate_dv d_v
    label_max_iter: int = 30


def alpha_q(a: float) -> int:
    """round_half_even(256 a), the fixed-point weighting factor (Python's
    round() rounds half to even)."""
    return int(round(a * 256.0))


class Network:
    """Float32 master parameters, the BF16 blob the kernels read, Adam state."""

    def __init__(self, device="cuda", seed: int = 0, alpha_default: float = 1.5):
        import torch

        rng = np.random.default_rng(seed)
        w1 = rng.standard_normal((64, 8)) * math.sqrt(2.0 / 8)
        w2 = rng.standard_normal((64, 64)) * math.sqrt(2.0 / 64)
        w3 = rng.standard_normal((2, 64)) * 0.01
        b = np.zeros(64 + 64)
        b3 = np.array([alpha_default, 0.0])
        master = np.concatenate([w1.ravel(), w2.ravel(), w3.ravel(), b, b3]).astype(np.float32)
        self.device = device
        self.master = torch.tensor(master, device=device)
        self.blob = torch.zeros(fwbf.MLP_BLOB_BYTES, dtype=torch.uint8, device=device)
        self.grad = torch.zeros(fwbf.MLP_PARAMS, dtype=torch.float32, device=device)
        self.m = torch.zeros_like(self.grad)
        self.v = torch.zeros_like(self.grad)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step = 0
        fwbf.fwbf_mlp_pack(self.master, self.blob)

    def set_master(self, master: np.ndarray):
        import torch

        self.master.copy_(torch.as_tensor(np.asarray(master, dtype=np.float32)))
        fwbf.fwbf_mlp_pack(self.master, self.blob)

    def save(self, path: str, **meta):
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        np.savez(path, master=self.master.cpu().numpy(), m=self.m.cpu().numpy(), v=self.v.cpu().numpy(),
                 step=self.step, **{k: np.asarray(v) for k, v in meta.items()})

    def load(self, path: str):
        import torch

        d = np.load(path)
        self.set_master(d["master"])
        if "m" in d:
            self.m.copy_(torch.as_tensor(d["m"]))
            self.v.copy_(torch.as_tensor(d["v"]))
            self.step = int(d["step"])
        return d

    def forward(self, x):
        import torch

        out = torch.empty((x.shape[0], 2), dtype=torch.float32, device=x.device)
        fwbf.fwbf_mlp_forward(self.blob, x.contiguous(), out)
        return out

    def train_epoch(self, X, T, batch: int = 8192, lr: float = 1e-3, perm=None):
        """One pass over (X, T) in mini-batches; returns the mean loss."""
        import torch

        n = X.shape[0]
        order = perm if perm is not None else torch.arange(n, device=X.device)
        total = 0.0
        for s0 in range(0, n, batch):
            idx = order[s0:s0 + batch]
            xb, tb = X[idx].contiguous(), T[idx].contiguous()
            self.loss.zero_()
            fwbf.fwbf_mlp_grad(self.blob, xb, tb, xb.shape[0], self.grad, self.loss)
            self.step += 1
            fwbf.fwbf_mlp_adam(self.master, self.blob, self.grad, self.m, self.v, self.step, lr)
            total += self.loss.item() * xb.shape[0]
        return total / max(n, 1)


def unpack_bits_torch(bits, N):
    import torch

    zb = bits.view(torch.uint8)
    z = ((zb.unsqueeze(-1) >> torch.arange(8, device=bits.device, dtype=torch.uint8)) & 1).reshape(bits.shape[0], -1)
    return z[:, :N]


def frame_ok(bits, iters, c):
    """Decoded to the transmitted codeword (converged and equal)."""
    return (iters >= 0) & (unpack_bits_torch(bits, c.shape[1]) == c).all(dim=1)


def label_schedules(code, q, c, sch: Schedule, chunk: int = 1 << 18):
    """Greedy per-pass labels on the GPU.  Returns int32 tensors
    (A, T) [F][label_max_iter] of the labelled alpha_q / theta_q."""
    import torch

    dev = q.device
    F = q.shape[0]
    K = sch.label_max_iter
    aq0 = alpha_q(sch.alpha_default)
    A = torch.full((F, K), aq0, dtype=torch.int32, device=dev)
    T = torch.zeros((F, K), dtype=torch.int32, device=dev)
    grid = [(alpha_q(a), int(round(t * 256))) for a in sch.grid_alpha for t in sch.grid_theta]
    dflt = grid.index((aq0, 0))
    active = torch.arange(F, device=dev)
    for k in range(sch.k_learn):
        if active.numel() == 0:
            break
        best = torch.full((active.numel(),), 1 << 20, dtype=torch.int64, device=dev)
        best_g = torch.full((active.numel(),), dflt, dtype=torch.int64, device=dev)
        for s0 in range(0, active.numel(), chunk):
            idx = active[s0:s0 + chunk]
            qa = q[idx].contiguous()
            ca = c[idx]
            scores = []
            for g, (ga, gt) in enumerate(grid):
                a_s = A[idx].clone()
                t_s = T[idx].clone()
                a_s[:, k] = ga
                t_s[:, k] = gt
                bits, iters = code.outputs(idx.numel(), dev)
                fwbf.fwbf_decode_sched(code.handle, qa, K, a_s, t_s, bits, iters)
                ok = frame_ok(bits, iters, ca)
                sc = torch.where(ok, iters.to(torch.int64), torch.full_like(iters, 1 << 20, dtype=torch.int64))
                scores.append(sc * 64 + (0 if g == dflt else 1))  # ties keep the default
            S = torch.stack(scores, dim=1)
            v, gi = S.min(dim=1)
            best[s0:s0 + idx.numel()] = v // 64
            best_g[s0:s0 + idx.numel()] = gi
        ga = torch.tensor([g[0] for g in grid], dtype=torch.int32, device=dev)
        gt = torch.tensor([g[1] for g in grid], dtype=torch.int32, device=dev)
        A[active, k] = ga[best_g]
        T[active, k] = gt[best_g]
        # frames solved within k + 1 passes, or unsolvable by any grid point, are done
        keep = (best > k + 1) & (best < (1 << 20))
        active = active[keep]
    return A, T


def training_set(code, q, A, T, sch: Schedule):
    """Features along the labelled trajectories and the matching targets
    (alpha, theta / 16) for every pass each frame runs (k < k_learn)."""
    import torch

    dev = q.device
    F = q.shape[0]
    feat = torch.zeros((F, sch.k_learn, fwbf.MLP_IN), dtype=torch.float32, device=dev)
    bits, iters = code.outputs(F, dev)
    fwbf.fwbf_decode_sched(code.handle, q, sch.label_max_iter, A, T, bits, iters, out_feat=feat)
    passes = torch.where(iters >= 0, iters, torch.full_like(iters, sch.k_learn)).clamp(max=sch.k_learn)
    mask = torch.arange(sch.k_learn, device=dev)[None, :] < passes[:, None]
    X = feat[mask]
    tgt = torch.stack([A[:, :sch.k_learn].float() / 256.0, T[:, :sch.k_learn].float() / 256.0 / 16.0], dim=-1)
    Y = tgt[mask]
    return X.contiguous(), Y.contiguous()


def wilson(k: int, n: int, z: float = 1.96):
    if n == 0:
        return (0.0, 1.0)
    p = k / n
    d = 1 + z * z / n
    cpt = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return (max(0.0, cpt - h), min(1.0, cpt + h))


def evaluate(code, q, c, net: Network | None, sch: Schedule, max_iter: int = 100, reps: int = 3):
    """FER (95% Wilson interval), bit errors, passes and decode time of the
    learned decoder (net given) or of plain FWBF (net None)."""
    import torch

    F = q.shape[0]
    dev = q.device
    bits, iters = code.outputs(F, dev)
    st = torch.cuda.current_stream()

    def run():
        if net is None:
            fwbf.fwbf_decode(code.handle, q, max_iter, sch.alpha_default, bits, iters)
        else:
            fwbf.fwbf_decode_learned(code.handle, q, max_iter, sch.k_learn, sch.alpha_default, net.blob, bits,
                                     iters, gate_dv=sch.gate_dv)

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        run()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ok = frame_ok(bits, iters, c)
    fe = int((~ok).sum().item())
    be = int((unpack_bits_torch(bits, c.shape[1]) != c).sum().item())
    passes = torch.where(iters >= 0, iters, torch.full_like(iters, max_iter)).float().mean().item()
    return {"frames": F, "frame_errors": fe, "fer": fe / F, "fer_ci95": wilson(fe, F),
            "ber": be / (F * c.shape[1]), "avg_passes": passes, "decode_ms": ms}


def make_frames(code_h, enc, F, ebn0_list, seed, device):
    """Seeded frames spread evenly over the Eb/N0 points; returns (q, c)."""
    import torch

    from .inputs.channel import bpsk_awgn_torch, random_codewords_torch

    per = [F // len(ebn0_list) + (1 if i < F % len(ebn0_list) else 0) for i in range(len(ebn0_list))]
    qs, cs = [], []
    for i, (eb, n) in enumerate(zip(ebn0_list, per)):
        _, c = random_codewords_torch(enc, n, seed=seed * 131 + i, device=device)
        y = bpsk_awgn_torch(c, eb, enc.rate, seed=seed * 131 + i)
        qs.append(fwbf.quantize(y.contiguous()))
        cs.append(c)
    return torch.cat(qs).contiguous(), torch.cat(cs)


def train_pipeline(code, enc, train_frames: int, ebn0_list, sch: Schedule, epochs: int = 4, seed: int = 1,
                   lr: float = 2e-3, log=print, oversample: int = 1):
    """Labels -> features -> training, all on the GPU.  Returns the network and
    a summary.  oversample > 1 repeats every sample whose label differs from
    the default that many times (the labels are mostly the default)."""
    import torch

    t0 = time.time()
    q, c = make_frames(code, enc, train_frames, ebn0_list, seed, "cuda")
    A, T = label_schedules(code, q, c, sch)
    torch.cuda.synchronize()
    t_label = time.time() - t0
    X, Y = training_set(code, q, A, T, sch)
    if oversample > 1:
        rare = (Y[:, 0] != alpha_q(sch.alpha_default) / 256.0) | (Y[:, 1] != 0.0)
        X = torch.cat([X] + [X[rare]] * (oversample - 1)).contiguous()
        Y = torch.cat([Y] + [Y[rare]] * (oversample - 1)).contiguous()
    changed = float(((A[:, :sch.k_learn] != alpha_q(sch.alpha_default)) | (T[:, :sch.k_learn] != 0)).float().mean())
    net = Network(seed=seed, alpha_default=sch.alpha_default)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(X.shape[0], device="cuda", generator=g)
        losses.append(net.train_epoch(X, Y, lr=lr, perm=perm))
        log(f"epoch {ep}: loss {losses[-1]:.5f}")
    return net, {"label_seconds": t_label, "samples": int(X.shape[0]), "labels_changed_frac": changed,
                 "losses": losses, "train_seconds": time.time() - t0}


def evaluate_batched(code, q, c, net: Network | None, sch: Schedule, max_iter: int = 100, reps: int = 3,
                     warps_per_cta: int = 16):
    """As evaluate(), through one graph-captured batched launch (the learned
    network, if given, runs inside the batch kernel)."""
    import torch

    F = q.shape[0]
    bits, iters = code.outputs(F, q.device)
    job = (code.handle, q, max_iter, sch.alpha_default, bits, iters)
    if net is not None:
        job = job + (net.blob, sch.k_learn, sch.gate_dv)
    batch = fwbf.fwbf_batch_create([job], warps_per_cta=warps_per_cta, packed=2)
    s = torch.cuda.Stream()
    try:
        with torch.cuda.stream(s):
            fwbf.fwbf_decode_batch(batch, s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            fwbf.fwbf_decode_batch(batch, s)
        # replay() launches on the current stream: time it there
        with torch.cuda.stream(s):
            g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                g.replay()
            e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
    finally:
        fwbf.fwbf_batch_destroy(batch)
    ok = frame_ok(bits, iters, c)
    fe = int((~ok).sum().item())
    be = int((unpack_bits_torch(bits, c.shape[1]) != c).sum().item())
    passes = torch.where(iters >= 0, iters, torch.full_like(iters, max_iter)).float().mean().item()
    return {"frames": F, "frame_errors": fe, "fer": fe / F, "fer_ci95": wilson(fe, F),
            "ber": be / (F * c.shape[1]), "avg_passes": passes, "decode_ms": ms}


def main():
    """Default: EG(1023,781), 3.0-4.5 dB; autotune (p, alpha) at 4 dB, label
    and train on seeded frames, evaluate plain (paper setting), tuned plain and
    learned (batched, graph-captured) on held-out frames.  --code / --ebn0 /
    --p-ref / --tune-ebn0 select another cyclic code and channel range."""
    import argparse
    import json

    import torch

    from . import autotune
    from .inputs import Encoder, make_code

    ap = argparse.ArgumentParser(description="train and evaluate the learned FWBF schedule on a cyclic code")
    ap.add_argument("--code", default="eg1023")
    ap.add_argument("--ebn0", default="3.0,3.5,4.0,4.5", help="comma-separated Eb/N0 points (dB)")
    ap.add_argument("--p-ref", type=int, default=31, help="the paper-setting block length of the comparison")
    ap.add_argument("--tune-ebn0", type=float, default=4.0)
    ap.add_argument("--train-frames", type=int, default=1 << 22)
    ap.add_argument("--eval-frames", type=int, default=1 << 18, help="held-out frames per Eb/N0 point")
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--k-learn", type=int, default=8)
    ap.add_argument("--out", default=None, help="weights file (default: weights/fwbf_mlp_<code>.npz)")
    ap.add_argument("--report", default=None)
    ap.add_argument("--weights", default=None, help="evaluate these weights instead of training")
    ap.add_argument("--oversample", type=int, default=1, help="repeat non-default labels this many times")
    ap.add_argument("--gate-dv", default="6",
                    help="comma-separated gates: the network runs on passes with W_k >= gate * d_v")
    args = ap.parse_args()
    gates = tuple(int(x) for x in args.gate_dv.split(","))
    torch.cuda.set_device(0)
    h = make_code(args.code)
    enc = Encoder(h)
    ebn0 = tuple(float(x) for x in args.ebn0.split(","))
    out_path = args.out or weights_path(args.code)
    tune = autotune.tune_code(h, enc, args.tune_ebn0, p_ref=args.p_ref, alpha_ref=1.5, frames=1 << 16)
    p_star, a_star = tune["choice"]["p"], tune["choice"]["alpha"]
    print(json.dumps({"autotune": tune["choice"], "reference": tune["reference"]}), flush=True)
    sch = Schedule(alpha_default=a_star, k_learn=args.k_learn)
    code = fwbf.Code.from_parity_check(h, p_star)
    if args.weights:
        net = Network(alpha_default=sch.alpha_default)
        meta = net.load(args.weights)
        summary = {"weights": os.path.basename(args.weights), "seg_len": int(meta["seg_len"])}
        if int(meta["seg_len"]) != p_star or float(meta["alpha_default"]) != a_star:
            p_star, a_star = int(meta["seg_len"]), float(meta["alpha_default"])
            sch = Schedule(alpha_default=a_star, k_learn=int(meta["k_learn"]))
            code = fwbf.Code.from_parity_check(h, p_star)
    else:
        net, summary = train_pipeline(code, enc, args.train_frames, ebn0, sch, epochs=args.epochs,
                                      log=lambda m: print(m, flush=True), oversample=args.oversample)
        net.save(out_path, seg_len=p_star, k_learn=sch.k_learn, alpha_default=sch.alpha_default)
    res = {"code": args.code, "autotune": tune, "train": summary, "seg_len": p_star, "alpha": a_star,
           "k_learn": sch.k_learn}
    paper = Schedule(alpha_default=1.5, k_learn=sch.k_learn)
    code31 = fwbf.Code.from_parity_check(h, args.p_ref)
    for eb in ebn0:
        q, c = make_frames(code, enc, args.eval_frames, (eb,), seed=777, device="cuda")
        point = {f"plain_p{args.p_ref}": evaluate(code31, q, c, None, paper),
                 "plain_tuned": evaluate(code, q, c, None, sch)}
        for g in gates:
            key = "learned_batched" if len(gates) == 1 else f"learned_batched_g{g}"
            point[key] = evaluate_batched(code, q, c, net, dataclasses.replace(sch, gate_dv=g))
        res[f"{eb}dB"] = point
        print(json.dumps({f"{eb}dB": res[f"{eb}dB"]}), flush=True)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
