"""The paper's delay model of the bit choice in a partially parallel hardware
decoder (Sec. IV, Eq. 2 and Eq. 3), as plain formulas.

2q metric values are computed per clock (N / 2q clocks for all N), and a
pipelined comparator network of log2(2q) stages takes the maximum of each
group of 2q values.  FWBF chooses its flips as the metric blocks stream
through the network (Eq. 3); lambda-largest selection (MLP-WBF) needs lambda
global maxima one after another, each a full sweep plus log2(N / 2q) further
clocks to reduce the local maxima (Eq. 2).  Clock counts are whole cycles:
N / 2q and the logarithms round up.  This models the paper's hardware; the
GPU decoder does not follow it.
"""
from __future__ import annotations

import math


def _clog2(x: int) -> int:
    return max(0, math.ceil(math.log2(x))) if x > 1 else 0


def sweep_clocks(N: int, two_q: int) -> int:
    """N / 2q: clocks to compute all N metrics, 2q per clock."""
    return -(-N // two_q)


def fwbf_choice_clocks(N: int, two_q: int) -> int:
    """Eq. 3: log2(2q) + N / 2q clocks per iteration for FWBF's bit choice."""
    return _clog2(two_q) + sweep_clocks(N, two_q)


def lambda_choice_clocks(N: int, two_q: int, lam: int) -> int:
    """Eq. 2: lambda (log2(2q) + N / 2q + log2(N / 2q)) clocks per iteration
    for choosing the lambda largest metrics one after another."""
    return lam * (_clog2(two_q) + sweep_clocks(N, two_q) + _clog2(sweep_clocks(N, two_q)))
