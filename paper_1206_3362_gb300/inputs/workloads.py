"""Named synthetic workloads: the codes, channel points and decoder settings the
decoder is tested and measured on.  Each entry states its recipe in full."""
from __future__ import annotations

import dataclasses
import functools

from .codes import eg2_cyclic, random_qc, random_regular


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    code: str            # key into make_code
    ebn0_db: tuple       # Eb/N0 points
    frames: int          # frames per point
    max_iter: int
    seg_len: int         # p, the block length of the partially parallel bit-choose
    codeword: str        # "zero" or "random" (seeded info bits, systematic encoding)
    alpha: float = 1.0   # IMWBF weighting factor of Eq. 1


CODE_SEED = 20120615


@functools.lru_cache(maxsize=None)
def make_code(key: str):
    if key == "rand504":      # (3,6)-regular, N=504, M=252
        return random_regular(504, 3, 6, seed=CODE_SEED)
    if key == "rand2016":     # (3,6)-regular, N=2016, M=1008
        return random_regular(2016, 3, 6, seed=CODE_SEED + 1)
    if key == "eg255":        # EG(2,2^4): (255,175)
        return eg2_cyclic(4)
    if key == "eg1023":       # EG(2,2^5): (1023,781)
        return eg2_cyclic(5)
    if key == "eg4095":       # EG(2,2^6): (4095,3367)
        return eg2_cyclic(6)
    if key == "eg15":         # EG(2,2^2): (15,7), for hand-checked traces
        return eg2_cyclic(2)
    if key == "qc8192":       # column weight 4, row weight 32, Z = 256
        return random_qc(256, 4, 32, seed=CODE_SEED + 2, weight=1)
    if key == "qc16384":      # 2 x 32 blocks of weight-2 circulants, Z = 512
        return random_qc(512, 2, 32, seed=CODE_SEED + 3, weight=2)
    raise KeyError(key)


WORKLOADS = {
    "rand504_4dB": Workload("rand504_4dB", "rand504", (4.0,), 1000, 50, 32, "zero"),
    "eg1023_sweep": Workload("eg1023_sweep", "eg1023",
                             tuple(3.0 + 0.25 * i for i in range(9)), 1 << 20, 100, 31, "random"),
    "eg1023_4dB": Workload("eg1023_4dB", "eg1023", (4.0,), 1 << 20, 100, 31, "random"),
}
