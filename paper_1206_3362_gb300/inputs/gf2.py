"""GF(2) linear algebra for building inputs: rank of H and a systematic encoder.

The encoder turns seeded information bits into codewords (H c = 0), which the
channel model then maps to BPSK/AWGN values.  It is input generation only.
"""
from __future__ import annotations

import numpy as np

from .codes import ParityCheck


def _packed(h: ParityCheck) -> np.ndarray:
    words = (h.N + 63) // 64
    a = np.zeros((h.M, words), dtype=np.uint64)
    w = h.cols // 64
    b = (h.cols % 64).astype(np.uint64)
    np.bitwise_xor.at(a, (h.rows, w), np.left_shift(np.uint64(1), b))
    return a


def gf2_rref(h: ParityCheck):
    """Reduced row-echelon form of H over GF(2) (rows bit-packed, 64 per word).

    Returns (R, pivots): R holds the rank-many non-zero rows and pivots[i] is the
    column of row i's leading one; every pivot column is zero in the other rows.
    """
    a = _packed(h)
    r = 0
    pivots = []
    for col in range(h.N):
        w, b = divmod(col, 64)
        bit = np.uint64(1) << np.uint64(b)
        cand = np.flatnonzero(a[r:, w] & bit)
        if cand.size == 0:
            continue
        p = r + int(cand[0])
        if p != r:
            a[[r, p]] = a[[p, r]]
        hit = (a[:, w] & bit) != 0
        hit[r] = False
        a[hit] ^= a[r]
        pivots.append(col)
        r += 1
        if r == h.M:
            break
    return a[:r], pivots


def gf2_rank(h: ParityCheck) -> int:
    return len(gf2_rref(h)[1])


def _unpack(rows: np.ndarray, n: int) -> np.ndarray:
    bits = np.unpackbits(rows.view(np.uint8), axis=1, bitorder="little")
    return bits[:, :n]


class Encoder:
    """Systematic encoder: the K = N - rank(H) non-pivot columns carry the
    information bits; each pivot bit is the XOR of the information bits its
    reduced row selects, which makes every row of H check to zero."""

    def __init__(self, h: ParityCheck):
        rref, pivots = gf2_rref(h)
        self.N = h.N
        self.rank = len(pivots)
        self.K = h.N - self.rank
        self.parity_pos = np.asarray(pivots, dtype=np.int64)
        mask = np.ones(h.N, dtype=bool)
        mask[self.parity_pos] = False
        self.info_pos = np.flatnonzero(mask)
        dense = _unpack(rref, h.N)
        self.A = dense[:, self.info_pos].astype(np.float64)  # rank x K

    @property
    def rate(self) -> float:
        return self.K / self.N

    def encode(self, u: np.ndarray) -> np.ndarray:
        """u: uint8 [F][K] information bits -> uint8 [F][N] codewords."""
        u = np.asarray(u, dtype=np.uint8)
        c = np.zeros((u.shape[0], self.N), dtype=np.uint8)
        c[:, self.info_pos] = u
        par = (u.astype(np.float64) @ self.A.T).astype(np.int64) & 1
        c[:, self.parity_pos] = par.astype(np.uint8)
        return c
