"""Throughput benchmark: FWBF decoding of EG(1023,781) frames on GB300.

One step = one pass of the whole decoding path over one batch: int8
quantisation of the float channel values, then FWBF decoding of every frame
(initialisation, syndrome, metric of Eq. 1, block arg-max, flips, stop test)
through the C ABI.  Inputs are synthetic (seeded random information bits,
systematic encoding, BPSK over AWGN) and already resident in HBM; they are far
larger than L2 (4.3 GB of float32 per step), so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  --impl reference times the CPU oracle on the host cores
on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import atexit
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "decoded info Gb/s on 1 GB300 at matched FER: learned+batched vs plain FWBF"
SM_COUNT = 152
INT_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0

WORKLOAD = dict(code="eg1023", ebn0_db=4.0, frames=1 << 20, max_iter=100, seg_len=31, alpha=1.5)

# DRAM bytes (read + write) per frame of the decode kernel from one ncu capture
# of DECODE_KERNEL (131,072 frames of this workload; scaled by frames, since
# traffic is the frame bytes in and the decisions out); see
# profiles/fwbf_decode_i8_eg1023_4dB.md.  Set to None when the kernel changes.
DECODE_TRAFFIC_BYTES_PER_FRAME = (134.140928e6 + 8.588800e6) / 131072
DECODE_KERNEL = "fwbf_decode_i8_cyclic_kernel<4, 2, true>"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=WORKLOAD["frames"])
    ap.add_argument("--no-peak", action="store_true", help="skip the integer issue-rate measurement")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="eg1023", choices=["eg1023", "batched4"],
                    help="eg1023: EG(1023,781) at 4 dB (default); batched4: four codes in one graph-captured launch")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the autotuned and learned batched forms on the same frames")
    return ap.parse_args()


def workload_config(frames):
    w = WORKLOAD
    return {
        "workload": f"EG(1023,781) FWBF int8, {frames} frames/step at Eb/N0 {w['ebn0_db']} dB "
                    f"(a point of the 3.0-5.0 dB sweep), random info bits, p={w['seg_len']}, "
                    f"K_max={w['max_iter']}, alpha={w['alpha']}",
        "code": "EG(2,2^5) type-I cyclic (1023,781)",
        "frames_per_step": frames,
        "ebn0_db": w["ebn0_db"],
        "seg_len": w["seg_len"],
        "max_iter": w["max_iter"],
        "alpha": w["alpha"],
        "l2": "inputs larger than L2 (no flush)",
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms from start()
    to stop().  begin() and end() mark the timed region on the host clock; the
    summary keeps the samples stamped inside it (every sample, and says so,
    when none is)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
            atexit.register(self._kill)  # never outlive the benchmark, even after an error
        except (OSError, FileNotFoundError):
            self.proc = None

    def _kill(self):
        if self.proc is not None and self.proc.poll() is None:
            self.proc.terminate()
            self.proc.wait()

    def begin(self):
        self.t0 = datetime.datetime.now()

    def end(self):
        self.t1 = datetime.datetime.now()

    @staticmethod
    def parse(text):
        """(timestamp or None, sm MHz, max sm MHz, active reasons) per row."""
        out = []
        for line in text.splitlines():
            r = [x.strip() for x in line.split(",")]
            if len(r) < 10:
                continue
            try:
                sm, mx = float(r[2]), float(r[3])
            except ValueError:
                continue
            try:
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                ts = None
            active = [n for n, v in zip(ClockSampler.REASONS, r[6:10]) if v.lower() == "active"]
            out.append((ts, sm, mx, active))
        return out

    def summarise(self, rows):
        window = "timed region"
        use = rows
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if r[0] is not None and self.t0 <= r[0] <= self.t1]
            if inside:
                use = inside
            else:
                window = "whole run (no sample stamped inside the timed region)"
        else:
            window = "whole run"
        reasons = sorted({n for r in use for n in r[3]})
        return {"sm_mhz": statistics.median(r[1] for r in use) if use else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "reasons": reasons, "samples": len(use), "window": window}

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = self.parse(self.tmp.read())
        os.unlink(self.tmp.name)
        return self.summarise(rows)


def algorithmic_ops(iters, max_iter, E, N, B):
    """Integer work the method defines for a batch: per frame one
    initialisation (2E + N: the weights and the syndrome) and, per flip pass,
    2E + N + B (syndrome and metric over every edge, one compare per bit, one
    flip test per block).  A frame that fails runs max_iter passes."""
    import torch

    passes = torch.where(iters < 0, torch.full_like(iters, max_iter), iters).to(torch.int64).sum().item()
    return iters.numel() * (2 * E + N) + passes * (2 * E + N + B)


def run_reference(args):
    """The CPU oracle, as it stands, on the machine's host cores: each step decodes
    a bounded sample of the workload's frames (host-generated, same recipe)."""
    import numpy as np

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1206_3362_gb300.inputs import Encoder, bpsk_awgn, make_code, random_codewords

    w = WORKLOAD
    h = make_code(w["code"])
    enc = Encoder(h)
    sample = 1024
    _, c = random_codewords(enc, sample, seed=2024)
    q = oracle.quantize(bpsk_awgn(c, w["ebn0_db"], enc.rate, seed=2024))
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.fwbf_i8_threaded(h, w["seg_len"], q[:threads], w["max_iter"], w["alpha"], threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.fwbf_i8_threaded(h, w["seg_len"], q, w["max_iter"], w["alpha"], threads=threads)
    dt = time.perf_counter() - t0
    value = sample * args.steps * enc.K / dt / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gb/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
        "data": "synthetic", "config": workload_config(sample),
        "cpu_baseline": {"value": value, "unit": "Gb/s", "cores": threads, "kind": "oracle",
                         "sample": f"{sample} frames per step of the same workload, host-generated"},
        "e2e": {"value": value, "unit": "Gb/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched4":
        run_batched4(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1206_3362_gb300 import fwbf
    from paper_1206_3362_gb300.inputs import Encoder, make_code
    from paper_1206_3362_gb300.inputs.channel import bpsk_awgn_torch, random_codewords_torch
    from paper_1206_3362_gb300.sharding import frame_seed, max_over_ranks

    w = WORKLOAD
    F = args.frames
    h = make_code(w["code"])
    enc = Encoder(h)
    E, N = h.nnz, h.N
    # weak scaling: every rank makes and decodes its own batch of F frames
    seed = frame_seed(1000, rank)
    _, c = random_codewords_torch(enc, F, seed=seed, device=dev)
    y = bpsk_awgn_torch(c, w["ebn0_db"], enc.rate, seed=seed).contiguous()
    code = fwbf.Code.from_parity_check(h, w["seg_len"])
    B = code.info.n_blocks
    q = torch.empty((F, N), dtype=torch.int8, device=dev)
    bits, iters = code.outputs(F, dev)
    stream = torch.cuda.current_stream()

    def step():
        fwbf.fwbf_quantize(y, q, stream)
        fwbf.fwbf_decode(code.handle, q, w["max_iter"], w["alpha"], bits, iters, stream)

    # measured integer issue rate of this GPU (the roofline's measured denominator)
    peak_meas = fwbf.fwbf_peak_int_issue(1, 200.0, stream) / 1e12 if not args.no_peak else None

    clocks = ClockSampler(local)
    clocks.start()  # running before the timed region begins
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # timed region: K steps; events around every decode launch for the roofline
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    t_start.record(stream)
    for k in range(args.steps):
        fwbf.fwbf_quantize(y, q, stream)
        ev[k][0].record(stream)
        fwbf.fwbf_decode(code.handle, q, w["max_iter"], w["alpha"], bits, iters, stream)
        ev[k][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    clock_info = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    dec_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    ms = max_over_ranks(ms, device=dev)
    assert fwbf.fwbf_last_status(stream) == 0

    info_bits = F * enc.K * world * args.steps
    value = info_bits / (ms / 1e3) / 1e9
    it = iters
    fail = (it < 0).float().mean().item()
    conv_iters = it[it >= 0].float().mean().item() if (it >= 0).any() else float("nan")
    ops = algorithmic_ops(it, w["max_iter"], E, N, B)
    peak = SM_COUNT * INT_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    achieved = ops / (dec_ms / 1e3) / 1e12
    # frame error rate against the transmitted codewords
    zb = bits.view(torch.uint8)
    fe = 0
    for s0 in range(0, F, 1 << 16):
        z = ((zb[s0:s0 + (1 << 16)].unsqueeze(-1) >> torch.arange(8, device=dev, dtype=torch.uint8)) & 1)
        z = z.reshape(z.shape[0], -1)[:, :N]
        fe += (z != c[s0:s0 + (1 << 16)]).any(dim=1).sum().item()
    fer = fe / F

    result = {
        "metric": METRIC, "value": value, "unit": "Gb/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": workload_config(F), "fer": fer, "failed_frames": fail,
        "avg_passes_converged": conv_iters,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak,
                     "traffic": (DECODE_TRAFFIC_BYTES_PER_FRAME * F if DECODE_TRAFFIC_BYTES_PER_FRAME else None),
                     "algorithmic_bytes": F * (N + 4 * ((N + 31) // 32) + 4),
                     "kernel": DECODE_KERNEL, "decode_ms": dec_ms,
                     "peak_basis": "152 SMs x 128 int32 lanes x 2070 MHz (derived)",
                     "peak_measured": peak_meas, "frac_of_measured": achieved / peak_meas if peak_meas else None,
                     "peak_measured_basis": "fwbf_peak_int_issue(mix=1): logic ops and integer multiply-adds "
                                            "alternating, 64 warps/SM, on this GPU before the timed region"},
        "gpu_launches": 2 * args.steps,
        "clocks": clock_info,
    }

    if rank == 0 and not args.no_compare:
        result["comparison"] = compare_forms(fwbf, h, enc, q, c, w, F, fer, value, dev)
    if rank == 0 and not args.no_e2e:
        result["e2e"] = e2e(args, fwbf, code, y, w, F, enc, dev, stream)
    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(fwbf, h, enc, q, bits, iters, w)
    if rank == 0:
        print(json.dumps(result))
    code.close()
    if world > 1:
        dist.destroy_process_group()


BATCH_MIX = [("rand504", 32, 4), ("rand2016", 32, 2), ("eg4095", 63, 1), ("qc8192", 64, 1)]


def run_batched4(args):
    """Four codes of uneven N, M and weights (random (3,6) N=504 and N=2016,
    EG(4095,3367), QC N=8192 Z=256), frames 4:2:1:1 summing to 2^20 at 4 dB,
    decoded by one persistent launch captured in a CUDA graph; p, alpha,
    warps per CTA and packing from the autotuner."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1206_3362_gb300 import autotune, fwbf, learned
    from paper_1206_3362_gb300.inputs import Encoder, make_code
    from paper_1206_3362_gb300.inputs.channel import bpsk_awgn_torch, random_codewords_torch

    torch.cuda.set_device(0)
    total = args.frames
    jobs, keep, info_bits, tunes = [], [], 0, {}
    for i, (key, p_ref, share) in enumerate(BATCH_MIX):
        h = make_code(key)
        enc = Encoder(h)
        F = total * share // 8
        t = autotune.tune_code(h, enc, 4.0, p_ref=p_ref, alpha_ref=1.5, frames=1 << 14,
                               p_candidates=(4, 8, 16, 32, 64), alpha_candidates=(1.5, 2.0))
        p, a = t["choice"]["p"], t["choice"]["alpha"]
        tunes[key] = {"p": p, "alpha": a, "frames": F, "N": h.N, "K": enc.K}
        _, c = random_codewords_torch(enc, F, seed=300 + i, device="cuda")
        q = fwbf.quantize(bpsk_awgn_torch(c, 4.0, enc.rate, seed=300 + i).contiguous())
        code = fwbf.Code.from_parity_check(h, p)
        bits, iters = code.outputs(F)
        jobs.append((code.handle, q, 100, a, bits, iters))
        keep.append((code, q, c, bits, iters, enc))
        info_bits += F * enc.K
    shape, rows = autotune.tune_batch_shape(jobs)
    batch = fwbf.fwbf_batch_create(jobs, warps_per_cta=shape["warps_per_cta"], packed=shape["packed"])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fwbf.fwbf_decode_batch(batch, s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fwbf.fwbf_decode_batch(batch, s)
    clocks = ClockSampler(0)
    clocks.start()  # running before the timed region begins
    with torch.cuda.stream(s):
        for _ in range(max(3, args.warmup)):
            g.replay()
        torch.cuda.synchronize()
        clocks.begin()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(args.steps):
            g.replay()
        e1.record(s)
    torch.cuda.synchronize()
    clocks.end()
    clock_info = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    assert fwbf.fwbf_batch_status() == 0
    for (code, q, c, bits, iters, enc), key in zip(keep, tunes):
        tunes[key]["fer"] = float((~learned.frame_ok(bits, iters, c)).float().mean().item())
    fwbf.fwbf_batch_destroy(batch)
    print(json.dumps({
        "metric": METRIC, "value": info_bits / (ms / 1e3) / 1e9, "unit": "Gb/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
        "config": {"workload": "batched: rand(3,6) N=504 / N=2016, EG(4095,3367), QC N=8192 Z=256; frames "
                               "4:2:1:1 of %d at Eb/N0 4 dB, one graph-captured persistent launch" % total,
                   "codes": tunes, "batch_shape": shape, "l2": "inputs larger than L2 (no flush)"},
        "gpu_launches": args.steps, "clocks": clock_info}))


def compare_forms(fwbf, h, enc, q, c, w, F, fer_plain, gbps_plain, dev):
    """The same frames through the throughput forms: the autotuned plain
    decoder (FER-qualified p and alpha) and the learned schedule, each as one
    graph-captured batched launch.  Decoded info Gb/s here covers the decode
    only (the quantised frames are reused)."""
    import torch

    from paper_1206_3362_gb300 import autotune, learned

    out = {"plain_paper_setting": {"p": w["seg_len"], "alpha": w["alpha"], "fer": fer_plain,
                                   "gbps_with_quantise": gbps_plain}}
    tune = autotune.tune_code(h, enc, w["ebn0_db"], p_ref=w["seg_len"], alpha_ref=w["alpha"], frames=1 << 15)
    p_t, a_t = tune["choice"]["p"], tune["choice"]["alpha"]
    forms = [("plain_paper_setting", w["seg_len"], w["alpha"], None),
             ("tuned_batched", p_t, a_t, None)]
    if os.path.exists(learned.DEFAULT_WEIGHTS):
        net = learned.Network(alpha_default=a_t)
        meta = net.load(learned.DEFAULT_WEIGHTS)
        forms.append(("learned_batched", int(meta["seg_len"]), float(meta["alpha_default"]), net))
    for name, p, a, net in forms:
        code = fwbf.Code.from_parity_check(h, p)
        sch = learned.Schedule(alpha_default=a, k_learn=8)
        r = learned.evaluate_batched(code, q, c, net, sch, max_iter=w["max_iter"], reps=3)
        code.close()
        entry = out.setdefault(name, {})
        entry.update({"p": p, "alpha": a, "fer": r["fer"], "fer_ci95": r["fer_ci95"],
                      "avg_passes": r["avg_passes"], "decode_ms": r["decode_ms"],
                      "gbps_decode": F * enc.K / (r["decode_ms"] / 1e3) / 1e9})
    out["autotune"] = {"choice": tune["choice"], "calibration_frames": tune["frames"],
                       "reference_frame_errors": tune["reference"]["frame_errors"]}
    return out


def e2e(args, fwbf, code, y, w, F, enc, dev, stream):
    """Same metric through the public host-buffer entry point
    (fwbf_decode_host): every step copies the float channel values from pinned
    host memory, quantises, decodes and copies the decisions and pass counts
    back, chunks pipelined over two streams."""
    import torch

    y_host = y.cpu().pin_memory()
    bits_host = torch.empty((F, code.words), dtype=torch.int32).pin_memory()
    iters_host = torch.empty(F, dtype=torch.int32).pin_memory()

    def step():
        fwbf.fwbf_decode_host(code.handle, y_host, w["max_iter"], w["alpha"], bits_host, iters_host,
                              chunk_frames=1 << 15, stream=stream)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 5))
    t0.record(stream)
    for _ in range(steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    return {"value": F * enc.K * steps / (ms / 1e3) / 1e9, "unit": "Gb/s",
            "h2d_bytes_per_step": y_host.numel() * 4,
            "d2h_bytes_per_step": bits_host.numel() * 4 + iters_host.numel() * 4,
            "steps": steps, "ms_per_step": ms / steps, "api": "fwbf_decode_host (2-stream chunk pipeline)"}


def cpu_baseline(fwbf, h, enc, q, bits, iters, w):
    """The CPU oracle on the host cores, on a bounded sample of the same
    frames; also reports how many sampled frames the GPU matched bit-exactly."""
    import numpy as np

    import oracle

    sample = 16384  # about 25 s of CPU work on this workload
    qs = q[:sample].cpu().numpy()
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    bo, io, used = oracle.fwbf_i8_threaded(h, w["seg_len"], qs, w["max_iter"], w["alpha"], threads=threads)
    dt = time.perf_counter() - t0
    gb = bits[:sample].cpu().numpy().view(np.uint32)
    gi = iters[:sample].cpu().numpy()
    match = int(((gi == io) & (gb == bo).all(axis=1)).sum())
    one = 512
    t1 = time.perf_counter()
    oracle.fwbf_i8(h, w["seg_len"], qs[:one], w["max_iter"], w["alpha"])
    dt1 = time.perf_counter() - t1
    return {"value": sample * enc.K / dt / 1e9, "unit": "Gb/s", "cores": used, "kind": "oracle",
            "sample": f"first {sample} frames of the timed batch, decoded once ({dt:.1f} s wall)",
            "parity_sample_match": f"{match}/{sample}",
            "single_thread": {"value": one * enc.K / dt1 / 1e9, "unit": "Gb/s",
                              "sample": f"first {one} frames, one thread ({dt1:.2f} s)"}}


if __name__ == "__main__":
    main()
