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

    python -m paper_1206_3362_gb300.experiments tab1 [--frames N]
    python -m paper_1206_3362_gb300.experiments eg255 [--frames N]
"""
from __future__ import annotations

import json

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


def main():
    import argparse

    import torch

    import __graft_entry__

    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["tab1", "eg255"])
    ap.add_argument("--frames", type=int, default=None)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    __graft_entry__.build()
    torch.cuda.set_device(0)
    res = tab1(args.frames or (1 << 16)) if args.what == "tab1" else eg255(args.frames or (1 << 17))
    text = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
