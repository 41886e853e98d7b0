"""Throughput benchmark: FWBF decoding on GB300, learned + batched against plain.

The headline step is the learned + batched form on EG(1023,781) at Eb/N0 = 4 dB:
int8 quantisation of 2^20 frames of float channel values, then one
graph-captured batched launch of the FWBF decoder whose per-pass weighting
factor and threshold come from the learned network (plain FWBF as its
fallback).  Plain FWBF in the paper's setting (p = 31, alpha = 1.5) runs the
same frames beside it, timed the same way, with its FER; both forms' decoded
information Gb/s and FER are in the line.  Inputs are synthetic (seeded random
information bits, systematic encoding, BPSK over AWGN) and already resident in
HBM; they are far larger than L2 (4.3 GB of float32 per step), so no flush is
needed.  The line also carries the batched four-code workload (config 2) and
the learned + batched workload at scale (config 4), each timed in its own
window with its own clock record.

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
INT_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0

WORKLOAD = dict(code="eg1023", ebn0_db=4.0, frames=1 << 20, max_iter=100, seg_len=31, alpha=1.5)

# DRAM bytes (read + write) per frame of each decode kernel, from one ncu
# capture of that kernel on 131,072 frames of this workload (traffic is the
# frame bytes in and the decisions out, so it scales with frames); None when
# the kernel has changed since the capture.  The capture's command and figures
# are in profiles/ (fwbf_decode_kernels_eg1023_4dB.md).
TRAFFIC_BYTES_PER_FRAME = {"plain": (134.186496e6 + 8.260096e6) / 131072,  # 1,087 B
                           # (1,088 B per frame before the learned body took its frame
                           # statistics lazily; not captured since)
                           "learned": None}
NETWORK_FLOPS_PER_EVAL = 2 * (8 * 64 + 64 * 64 + 64 * 2)  # multiply-adds of 8 -> 64 -> 64 -> 2, x2


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=WORKLOAD["frames"])
    ap.add_argument("--no-peak", action="store_true", help="skip the integer issue-rate measurement")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the batched four-code and the at-scale workloads")
    ap.add_argument("--scale4-frames", type=int, default=1 << 22)
    return ap.parse_args(argv)


def workload_config(frames):
    w = WORKLOAD
    return {
        "workload": f"EG(1023,781) FWBF int8, {frames} frames/step at Eb/N0 {w['ebn0_db']} dB "
                    f"(a point of the 3.0-5.0 dB sweep), random info bits, K_max={w['max_iter']}: "
                    "learned + batched (value) against plain FWBF p=31, alpha=1.5 (plain_fwbf)",
        "code": "EG(2,2^5) type-I cyclic (1023,781)",
        "frames_per_step": frames,
        "ebn0_db": w["ebn0_db"],
        "max_iter": w["max_iter"],
        "l2": "inputs larger than L2 (no flush)",
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms from start()
    to stop().  begin() and end() mark the timed region on the host clock (or
    mark(name) / unmark(name) several named regions); summaries keep the
    samples stamped inside a region (every sample, and say so, when none is)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None
        self.t0 = self.t1 = None
        self.windows = {}
        self.rows = None

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

    def mark(self, name):
        self.windows[name] = [datetime.datetime.now(), None]

    def unmark(self, name):
        self.windows[name][1] = datetime.datetime.now()

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

    @staticmethod
    def window_summary(rows, t0, t1):
        window = "timed region"
        use = rows
        if t0 is not None and t1 is not None:
            inside = [r for r in rows if r[0] is not None and t0 <= r[0] <= t1]
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

    def summarise(self, rows):
        return self.window_summary(rows, self.t0, self.t1)

    def stop(self):
        """Stops sampling; returns the summary of the begin()/end() region."""
        if self.proc is None:
            self.rows = []
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.tmp.flush()
        self.tmp.seek(0)
        self.rows = self.parse(self.tmp.read())
        os.unlink(self.tmp.name)
        return self.summarise(self.rows)

    def window(self, name):
        """Summary of a named region (after stop())."""
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t0, t1 = self.windows.get(name, (None, None))
        return self.window_summary(self.rows, t0, t1)


def algorithmic_ops(iters, max_iter, E, N, B):
    """Integer work the method defines for a batch: per frame one
    initialisation (2E + N: the weights and the syndrome) and, per flip pass,
    2E + N + B (syndrome and metric over every edge, one compare per bit, one
    flip test per block).  A frame that fails is counted at max_iter passes."""
    import torch

    passes = torch.where(iters < 0, torch.full_like(iters, max_iter), iters).to(torch.int64).sum().item()
    return iters.numel() * (2 * E + N) + passes * (2 * E + N + B)


def pack_hard_decisions(q):
    """Bit-packed z_0 = (q < 0) of int8 frames, in the decoders' output layout
    (bit n in word n / 32, position n % 32)."""
    import torch

    F, N = q.shape
    words = (N + 31) // 32
    z = torch.zeros((F, words * 32), dtype=torch.int64, device=q.device)
    z[:, :N] = (q < 0).to(torch.int64)
    z = (z.reshape(F, words, 32) << torch.arange(32, device=q.device)).sum(dim=2)
    return torch.where(z >= (1 << 31), z - (1 << 32), z).to(torch.int32)  # the same 32 bits, signed


def executed_passes(fwbf, code, q, bits, iters, max_iter, alpha, z0=None):
    """Passes the plain decoder actually runs per frame.  A converged frame
    runs iters passes; a failing frame stops at the first pass that flips
    nothing (its decisions then stay the same for every larger pass limit) or
    at max_iter.  For the failing frames, decisions are recomputed under every
    pass limit m = 1 .. max_iter - 1: the frame's state settled at the smallest
    m from which they equal the final decisions for every larger limit, and it
    ran m + 1 passes (the last one finding no flip); a frame that never settles
    ran max_iter.  z0 (the failing frames' packed hard decisions, from q when
    None) tells a frame whose first pass flips nothing (m = 0: one pass).
    Returns a tensor of pass counts."""
    import torch

    passes = iters.clone().to(torch.int64)
    fail = torch.nonzero(iters < 0).flatten()
    if fail.numel() == 0:
        return passes
    qf = q[fail].contiguous()
    final = bits[fail]
    settled = torch.full((fail.numel(),), max_iter, dtype=torch.int64, device=q.device)
    b, i = code.outputs(fail.numel())
    for m in range(max_iter - 1, 0, -1):  # from the top: keep the smallest m of an unbroken run of equality
        fwbf.fwbf_decode(code.handle, qf, m, alpha, b, i)
        same = (b == final).all(dim=1)
        settled = torch.where(same & (settled == m + 1), torch.full_like(settled, m), settled)
    if z0 is None:
        z0 = pack_hard_decisions(qf)
    settled = torch.where((settled == 1) & (z0 == final).all(dim=1), torch.zeros_like(settled), settled)
    passes[fail] = torch.where(settled < max_iter, settled + 1, settled)
    return passes


def run_reference(args):
    """The CPU oracle, as it stands, on the machine's host cores: each step decodes
    a bounded sample of the workload's frames (host-generated, same recipe)."""
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
                         "sample": f"{sample} frames per step of the same workload, host-generated "
                                   "(plain FWBF p=31, alpha=1.5: the oracle of the method)"},
        "e2e": {"value": value, "unit": "Gb/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def frame_errors(bits, iters, c, N, chunk=1 << 16):
    """Frames not decoded to the transmitted codeword (or not converged)."""
    import torch

    zb = bits.view(torch.uint8)
    fe = 0
    for s0 in range(0, bits.shape[0], chunk):
        z = ((zb[s0:s0 + chunk].unsqueeze(-1) >> torch.arange(8, device=bits.device, dtype=torch.uint8)) & 1)
        z = z.reshape(z.shape[0], -1)[:, :N]
        fe += ((z != c[s0:s0 + chunk]).any(dim=1) | (iters[s0:s0 + chunk] < 0)).sum().item()
    return int(fe)


def timed(steps, stream, launch, step=None):
    """Runs `steps` steps on `stream`: step() (untimed part of the step, e.g.
    quantisation) then launch() between CUDA events.  Returns (whole-step ms,
    mean ms of the launches)."""
    import torch

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for k in range(steps):
        if step is not None:
            step()
        ev[k][0].record(stream)
        launch()
        ev[k][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), statistics.mean(a.elapsed_time(b) for a, b in ev)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return

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
    from paper_1206_3362_gb300 import autotune, fwbf, learned
    from paper_1206_3362_gb300.inputs import Encoder, make_code
    from paper_1206_3362_gb300.inputs.channel import bpsk_awgn_torch, random_codewords_torch
    from paper_1206_3362_gb300.sharding import frame_seed, max_over_ranks

    w = WORKLOAD
    F, K_max = args.frames, w["max_iter"]
    h = make_code(w["code"])
    enc = Encoder(h)
    E, N = h.nnz, h.N
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # weak scaling: every rank makes and decodes its own batch of F frames
    seed = frame_seed(1000, rank)
    _, c = random_codewords_torch(enc, F, seed=seed, device=dev)
    y = bpsk_awgn_torch(c, w["ebn0_db"], enc.rate, seed=seed).contiguous()
    q = torch.empty((F, N), dtype=torch.int8, device=dev)
    gs = torch.cuda.Stream(device=dev)  # every timed launch runs here (graphs need a side stream)

    # the learned form: the committed network with its block length and
    # weighting factor; the gate (passes that consult the network) from the
    # autotuner on separate calibration frames
    net = learned.Network(alpha_default=2.0)
    meta = net.load(learned.DEFAULT_WEIGHTS)
    p_l, a_l, k_l = int(meta["seg_len"]), float(meta["alpha_default"]), int(meta["k_learn"])
    code_l = fwbf.Code.from_parity_check(h, p_l)
    qcal, ccal = autotune.calibration_frames(h, enc, 1 << 18, w["ebn0_db"], seed=seed + 77, device=dev)
    gate = autotune.tune_gate(code_l, qcal, ccal, net, a_l, k_l, max_iter=K_max, reps=2)
    gate_dv = gate["choice"]
    del qcal, ccal
    bits_l, iters_l = code_l.outputs(F, dev)
    batch = fwbf.fwbf_batch_create([(code_l.handle, q, K_max, a_l, bits_l, iters_l, net.blob, k_l, gate_dv)],
                                   warps_per_cta=16, packed=2)
    with torch.cuda.stream(gs):
        fwbf.fwbf_quantize(y, q, gs)
        fwbf.fwbf_decode_batch(batch, gs)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        fwbf.fwbf_decode_batch(batch, gs)
    # plain FWBF in the paper's setting on the same frames
    code_p = fwbf.Code.from_parity_check(h, w["seg_len"])
    bits_p, iters_p = code_p.outputs(F, dev)

    def quantize():
        fwbf.fwbf_quantize(y, q, gs)

    def plain():
        fwbf.fwbf_decode(code_p.handle, q, K_max, w["alpha"], bits_p, iters_p, gs)

    # measured integer issue rate of this GPU (the roofline's measured denominator)
    peak_meas = fwbf.fwbf_peak_int_issue(1, 200.0, gs) / 1e12 if not args.no_peak else None

    clocks = ClockSampler(local)
    clocks.start()  # running before the timed regions begin
    steps, warm = args.steps, max(3, args.warmup)
    with torch.cuda.stream(gs):
        for _ in range(warm):
            quantize()
            graph.replay()
            quantize()
            plain()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks.begin()
        ms_l, dec_l = timed(steps, gs, graph.replay, step=quantize)
        clocks.end()
        if world > 1:
            dist.barrier()
        clocks.mark("plain")
        ms_p, dec_p = timed(steps, gs, plain, step=quantize)
        clocks.unmark("plain")
    clock_info = clocks.stop()
    if world > 1:
        dist.barrier()
    ms_l, ms_p = max_over_ranks(ms_l, device=dev), max_over_ranks(ms_p, device=dev)
    assert fwbf.fwbf_batch_status(gs) == 0 and fwbf.fwbf_last_status(gs) == 0

    info_bits = F * enc.K * world * steps
    value = info_bits / (ms_l / 1e3) / 1e9
    value_p = info_bits / (ms_p / 1e3) / 1e9
    fe_l, fe_p = frame_errors(bits_l, iters_l, c, N), frame_errors(bits_p, iters_p, c, N)

    # plain FWBF's roofline: the method's integer work, with failing frames
    # counted at K_max passes (the formula) and at the passes actually run
    B_p = code_p.info.n_blocks
    peak = sms * INT_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    ops_formula = algorithmic_ops(iters_p, K_max, E, N, B_p)
    run_passes = executed_passes(fwbf, code_p, q, bits_p, iters_p, K_max, w["alpha"])
    ops_run = F * (2 * E + N) + int(run_passes.sum().item()) * (2 * E + N + B_p)
    ach_f, ach_r = ops_formula / (dec_p / 1e3) / 1e12, ops_run / (dec_p / 1e3) / 1e12
    plain_roofline = {
        "bound": "alu", "unit": "Tops/s", "kernel": "fwbf_decode_i8_cyclic_kernel<4, 2, 0>", "decode_ms": dec_p,
        "achieved": ach_f, "frac": ach_f / peak, "achieved_run": ach_r, "frac_run": ach_r / peak,
        "peak": peak, "peak_basis": f"{sms} SMs x {INT_LANES_PER_SM} int32 lanes x {SM_MAX_MHZ:.0f} MHz (derived)",
        "peak_measured": peak_meas,
        "frac_of_measured": ach_f / peak_meas if peak_meas else None,
        "frac_run_of_measured": ach_r / peak_meas if peak_meas else None,
        "passes_formula": float(torch.where(iters_p < 0, torch.full_like(iters_p, K_max), iters_p).float().mean()),
        "passes_run": float(run_passes.float().mean()),
        "traffic": (TRAFFIC_BYTES_PER_FRAME["plain"] * F if TRAFFIC_BYTES_PER_FRAME["plain"] else None),
        "algorithmic_bytes": F * (N + 4 * ((N + 31) // 32) + 4),
    }

    # the learned kernel's work: the method's integer work (formula) plus the
    # network's multiply-adds, evaluations counted from a recording run (the
    # same decisions, checked)
    sched = torch.full((F, k_l, 2), -1, dtype=torch.int32, device=dev)
    feat = torch.zeros((F, k_l, fwbf.MLP_IN), dtype=torch.float32, device=dev)
    bits_r, iters_r = code_l.outputs(F, dev)
    fwbf.fwbf_decode_learned(code_l.handle, q, K_max, k_l, a_l, net.blob, bits_r, iters_r, out_sched=sched,
                             out_feat=feat, stream=gs, gate_dv=gate_dv)
    torch.cuda.synchronize()
    assert torch.equal(bits_r, bits_l) and torch.equal(iters_r, iters_l)
    dv = code_l.info.dv_max
    evals = int(((sched[:, :, 0] >= 0) & (torch.round(feat[:, :, 0] * N) >= gate_dv * dv)).sum().item())
    del sched, feat, bits_r, iters_r
    ops_l = algorithmic_ops(iters_l, K_max, E, N, code_l.info.n_blocks) + evals * NETWORK_FLOPS_PER_EVAL
    ach_l = ops_l / (dec_l / 1e3) / 1e12
    roofline = {
        "bound": "alu", "achieved": ach_l, "peak": peak, "unit": "Tops/s", "frac": ach_l / peak,
        "traffic": (TRAFFIC_BYTES_PER_FRAME["learned"] * F if TRAFFIC_BYTES_PER_FRAME["learned"] else None),
        "algorithmic_bytes": F * (N + 4 * ((N + 31) // 32) + 4),
        "kernel": "fwbf_decode_batch_kernel<true, true, true, 2> (one learned job)", "decode_ms": dec_l,
        "ops_basis": "method integer ops (init 2E+N per frame, 2E+N+B per pass, failures at K_max) + "
                     f"{NETWORK_FLOPS_PER_EVAL} flops per network evaluation",
        "peak_basis": plain_roofline["peak_basis"], "peak_measured": peak_meas,
        "frac_of_measured": ach_l / peak_meas if peak_meas else None,
        "peak_measured_basis": "fwbf_peak_int_issue(mix=1): logic ops and integer multiply-adds alternating, "
                               "64 warps/SM, on this GPU before the timed region",
    }

    result = {
        "metric": METRIC, "value": value, "unit": "Gb/s", "n_gpus": world, "steps": steps, "warmup": warm,
        "ms_per_step": ms_l / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int8", "data": "synthetic", "config": workload_config(F),
        "fer": fe_l / F, "fer_ci95": learned.wilson(fe_l, F),
        "learned_batched": {
            "p": p_l, "alpha_fallback": a_l, "k_learn": k_l, "gate_dv": gate_dv, "frame_errors": fe_l,
            "fer": fe_l / F, "fer_ci95": learned.wilson(fe_l, F), "gbps": value,
            "gbps_decode": F * enc.K * world / (dec_l / 1e3) / 1e9, "decode_ms": dec_l,
            "network_evals_per_frame": evals / F, "launch": "one graph-captured batched launch per step",
            "gate_tuning": gate},
        "plain_fwbf": {
            "p": w["seg_len"], "alpha": w["alpha"], "frame_errors": fe_p, "fer": fe_p / F,
            "fer_ci95": learned.wilson(fe_p, F), "gbps": value_p,
            "gbps_decode": F * enc.K * world / (dec_p / 1e3) / 1e9, "decode_ms": dec_p,
            "ms_per_step": ms_p / steps, "clocks": clocks.window("plain"), "roofline": plain_roofline},
        "speedup_vs_plain": value / value_p,
        "roofline": roofline,
        "gpu_launches": 2 * steps,
        "clocks": clock_info,
    }
    if rank == 0 and not args.no_e2e:
        result["e2e"] = e2e_learned(args, fwbf, code_l, net, y, F, enc, K_max, a_l, k_l, gate_dv, dev)
    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(h, enc, q, bits_p, iters_p, w)
    fwbf.fwbf_batch_destroy(batch)
    code_l.close()
    code_p.close()
    del y, q, c, bits_l, iters_l, bits_p, iters_p
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_configs:
        result["batched4"] = run_batched4(args)
        result["scale4"] = run_scale4(args)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


def e2e_learned(args, fwbf, code, net, y, F, enc, K_max, alpha, k_learn, gate_dv, dev, chunk=1 << 15):
    """The headline form end to end through the public API: every step copies
    the float channel values from pinned host memory, quantises them
    (fwbf_quantize), decodes them with the learned schedule
    (fwbf_decode_learned) and copies the decisions and pass counts back, in
    chunks alternating over two streams so that one chunk's copies overlap
    another's decoding."""
    import torch

    y_host = y.cpu().pin_memory()
    words = (y.shape[1] + 31) // 32
    bits_host = torch.empty((F, words), dtype=torch.int32).pin_memory()
    iters_host = torch.empty(F, dtype=torch.int32).pin_memory()
    streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    n = min(chunk, F)
    slots = [dict(y=torch.empty((n, y.shape[1]), dtype=torch.float32, device=dev),
                  q=torch.empty((n, y.shape[1]), dtype=torch.int8, device=dev),
                  bits=torch.empty((n, words), dtype=torch.int32, device=dev),
                  iters=torch.empty(n, dtype=torch.int32, device=dev)) for _ in range(2)]
    main = torch.cuda.current_stream(dev)

    def step():
        start = torch.cuda.Event()
        start.record(main)
        for s in streams:
            s.wait_event(start)
        for i, s0 in enumerate(range(0, F, n)):
            s, b = streams[i % 2], slots[i % 2]  # a slot is reused only on its own stream
            m = min(n, F - s0)
            with torch.cuda.stream(s):
                b["y"][:m].copy_(y_host[s0:s0 + m], non_blocking=True)
                fwbf.fwbf_quantize(b["y"][:m], b["q"][:m], s)
                fwbf.fwbf_decode_learned(code.handle, b["q"][:m], K_max, k_learn, alpha, net.blob, b["bits"][:m],
                                         b["iters"][:m], stream=s, gate_dv=gate_dv)
                bits_host[s0:s0 + m].copy_(b["bits"][:m], non_blocking=True)
                iters_host[s0:s0 + m].copy_(b["iters"][:m], non_blocking=True)
        for s in streams:
            done = torch.cuda.Event()
            done.record(s)
            main.wait_event(done)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 5))
    t0.record(main)
    for _ in range(steps):
        step()
    t1.record(main)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    return {"value": F * enc.K * steps / (ms / 1e3) / 1e9, "unit": "Gb/s",
            "h2d_bytes_per_step": y_host.numel() * 4,
            "d2h_bytes_per_step": bits_host.numel() * 4 + iters_host.numel() * 4,
            "steps": steps, "ms_per_step": ms / steps,
            "api": f"fwbf_quantize + fwbf_decode_learned (gate_dv {gate_dv}), pinned host buffers, "
                   f"{n}-frame chunks over 2 streams"}


def cpu_baseline(h, enc, q, bits, iters, w):
    """The CPU oracle (plain FWBF, the method) on the host cores, on a bounded
    sample of the same frames; also reports how many sampled frames the GPU's
    plain decoder matched bit-exactly."""
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
            "sample": f"first {sample} frames of the timed batch, plain FWBF p={w['seg_len']}, decoded once "
                      f"({dt:.1f} s wall)",
            "parity_sample_match": f"{match}/{sample}",
            "single_thread": {"value": one * enc.K / dt1 / 1e9, "unit": "Gb/s",
                              "sample": f"first {one} frames, one thread ({dt1:.2f} s)"}}


BATCH_MIX = [("rand504", 32, 4), ("rand2016", 32, 2), ("eg4095", 63, 1), ("qc8192", 64, 1)]


def run_batched4(args, total=1 << 20, steps=10):
    """Config 2: four codes of uneven N, M and weights (random (3,6) N=504 and
    N=2016, EG(4095,3367), QC N=8192 Z=256), frames 4:2:1:1 summing to 2^20 at
    4 dB, decoded by one persistent launch captured in a CUDA graph; p, alpha,
    warps per CTA and packing from the autotuner.  Its own clock window."""
    import torch

    from paper_1206_3362_gb300 import autotune, fwbf, learned
    from paper_1206_3362_gb300.inputs import Encoder, make_code
    from paper_1206_3362_gb300.inputs.channel import bpsk_awgn_torch, random_codewords_torch

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
    shape, _ = autotune.tune_batch_shape(jobs)
    batch = fwbf.fwbf_batch_create(jobs, warps_per_cta=shape["warps_per_cta"], packed=shape["packed"])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        fwbf.fwbf_decode_batch(batch, s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fwbf.fwbf_decode_batch(batch, s)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    with torch.cuda.stream(s):
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        clocks.begin()
        ms, dec = timed(steps, s, g.replay)
        clocks.end()
    clock_info = clocks.stop()
    assert fwbf.fwbf_batch_status(s) == 0
    for (code, q, c, bits, iters, enc), key in zip(keep, tunes):
        tunes[key]["fer"] = float((~learned.frame_ok(bits, iters, c)).float().mean().item())
    fwbf.fwbf_batch_destroy(batch)
    for k in keep:
        k[0].close()
    return {"workload": f"batched: rand(3,6) N=504 / N=2016, EG(4095,3367), QC N=8192 Z=256; frames 4:2:1:1 "
                        f"of {total} at Eb/N0 4 dB, one graph-captured persistent launch",
            "value": info_bits / (ms / steps / 1e3) / 1e9, "unit": "Gb/s", "steps": steps,
            "ms_per_step": ms / steps, "decode_ms": dec, "codes": tunes, "batch_shape": shape,
            "l2": "inputs larger than L2 (no flush)", "gpu_launches": steps, "clocks": clock_info}


def run_scale4(args):
    """Config 4: the rate-0.94 quasi-cyclic N=16384 code and EG(4095,3367),
    2^22 frames over 4.0-5.5 dB: plain FWBF (paper setting, one launch per code
    and point) against learned + batched (one graph-captured launch, autotuned
    block lengths, gates and CTA shape, the learned schedule on the EG code),
    on the same frames.  Its own clock window."""
    import torch

    from paper_1206_3362_gb300 import experiments

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    out = experiments.scale4(frames=args.scale4_frames, reps=2, clocks=clocks)
    clocks.stop()
    out["clocks_plain"] = clocks.window("plain")
    out["clocks_learned_batched"] = clocks.window("learned_batched")
    return out


if __name__ == "__main__":
    main()
