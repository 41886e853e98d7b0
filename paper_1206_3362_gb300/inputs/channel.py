"""BPSK over AWGN (Sec. II and V): s_n = 1 - 2 c_n, y = s + noise with
variance N0/2.  With unit symbol energy and code rate R = K/N the per-symbol
noise variance at a given Eb/N0 is sigma^2 = 1 / (2 R 10^(EbN0/10)).

Every draw is seeded: numpy's Philox counter-based generator keyed by
(seed, stream id) on the host, torch's seeded generator on the device.
"""
from __future__ import annotations

import math

import numpy as np


def awgn_sigma(ebn0_db: float, rate: float) -> float:
    return math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))


def rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, *stream])))


def random_codewords(encoder, n_frames: int, seed: int):
    """Seeded information bits and their systematic codewords."""
    u = rng(seed, 1).integers(0, 2, size=(n_frames, encoder.K), dtype=np.uint8)
    return u, encoder.encode(u)


def bpsk_awgn(c: np.ndarray, ebn0_db: float, rate: float, seed: int) -> np.ndarray:
    """float32 [F][N] channel values for codewords c (uint8 [F][N])."""
    sigma = awgn_sigma(ebn0_db, rate)
    noise = rng(seed, 2, int(round(ebn0_db * 1000))).standard_normal(c.shape, dtype=np.float32)
    s = 1.0 - 2.0 * c.astype(np.float32)
    return (s + np.float32(sigma) * noise).astype(np.float32)


def bpsk_awgn_torch(c, ebn0_db: float, rate: float, seed: int):
    """Device-side equivalent for large workloads: same recipe, torch's seeded
    generator on the tensor's device (different numbers than the host path)."""
    import torch

    g = torch.Generator(device=c.device)
    g.manual_seed(int(seed) * 1000003 + int(round(ebn0_db * 1000)))
    sigma = awgn_sigma(ebn0_db, rate)
    noise = torch.randn(c.shape, generator=g, device=c.device, dtype=torch.float32)
    return (1.0 - 2.0 * c.to(torch.float32)) + sigma * noise


def random_codewords_torch(encoder, n_frames: int, seed: int, device):
    """Seeded information bits and codewords built on the device: parity bits
    are an exact 0/1 matrix product reduced mod 2 (TF32 tensor-core inputs hold
    0 and 1 exactly and the fp32 sums stay below K < 2^24)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 7919 + 17)
    u = torch.randint(0, 2, (n_frames, encoder.K), generator=g, device=device, dtype=torch.uint8)
    a = torch.as_tensor(encoder.A.T, dtype=torch.float32, device=device)  # K x rank
    c = torch.zeros((n_frames, encoder.N), dtype=torch.uint8, device=device)
    info = torch.as_tensor(encoder.info_pos, device=device)
    par_pos = torch.as_tensor(encoder.parity_pos, device=device)
    c[:, info] = u
    chunk = 1 << 16
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        for s0 in range(0, n_frames, chunk):
            par = (u[s0:s0 + chunk].to(torch.float32) @ a).to(torch.int64) & 1
            c[s0:s0 + chunk, par_pos] = par.to(torch.uint8)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    return u, c
