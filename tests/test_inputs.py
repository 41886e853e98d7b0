"""Seeded input generators: code constructions and the channel model."""
import json
import math
import os

import numpy as np
import pytest

from paper_1206_3362_gb300.inputs import (Encoder, awgn_sigma, bpsk_awgn, eg2_cyclic, gf2_rank,
                                          make_code, random_codewords, random_qc, random_regular)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _paper():
    with open(os.path.join(GOLD, "paper_values.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("s,N,K", [tuple(v) for v in _paper()["code_parameters"]["eg"] if v[0] <= 5])
def test_eg_code_parameters(s, N, K):
    """EG(2,2^s) type-I codes have the (N, K) the paper quotes (Sec. IV-V):
    weights 2^s, RC constraint, and GF(2) rank N - K."""
    h = eg2_cyclic(s)
    assert h.N == N and h.M == N
    assert set(h.row_weights()) == {1 << s} and set(h.col_weights()) == {1 << s}
    assert h.max_row_overlap() == 1 and h.max_col_overlap() == 1
    assert not h.has_duplicates()
    assert N - gf2_rank(h) == K


@pytest.mark.slow
def test_eg4095_parameters():
    s, N, K = _paper()["code_parameters"]["eg"][3]
    h = eg2_cyclic(s)
    assert h.N == N and set(h.row_weights()) == {64}
    assert N - gf2_rank(h) == K


def test_eg_any_two_points_one_line():
    """In EG(2,2^s) two points lie on exactly one line; a line that misses the
    origin is a row of H.  So every pair of columns shares at most one row and
    the number of pairs covered is exactly M * C(2^s, 2)."""
    h = eg2_cyclic(4)
    H = h.dense().astype(np.int64)
    g = H.T @ H
    off = g[~np.eye(h.N, dtype=bool)]
    assert off.max() == 1
    assert off.sum() // 2 == h.M * (16 * 15 // 2)


@pytest.mark.parametrize("N,dv,dc", [(504, 3, 6), (2016, 3, 6), (120, 3, 6)])
def test_random_regular(N, dv, dc):
    h = random_regular(N, dv, dc, seed=5)
    assert set(h.col_weights()) == {dv} and set(h.row_weights()) == {dc}
    assert not h.has_duplicates()
    assert h.max_row_overlap() <= 1  # no 4-cycles
    h2 = random_regular(N, dv, dc, seed=5)
    assert np.array_equal(h.rows, h2.rows) and np.array_equal(h.cols, h2.cols)


def test_qc_code():
    h = make_code("qc8192")
    assert (h.N, h.M) == (8192, 1024)
    assert set(h.col_weights()) == {4} and set(h.row_weights()) == {32}
    assert h.max_row_overlap() <= 1 and not h.has_duplicates()
    # block structure: every Z x Z block is a circulant permutation
    Z = 256
    blk = (h.rows // Z) * 32 + (h.cols // Z)
    shift = (h.cols % Z - h.rows % Z) % Z
    for b in np.unique(blk):
        assert np.unique(shift[blk == b]).size == 1


def test_qc_weight2():
    h = random_qc(64, 2, 6, seed=3, weight=2)
    assert set(h.col_weights()) == {4} and set(h.row_weights()) == {12}
    assert h.max_row_overlap() <= 1


@pytest.mark.parametrize("key", ["eg255", "rand504", "qc8192"])
def test_encoder_codewords_check(key):
    h = make_code(key)
    enc = Encoder(h)
    u, c = random_codewords(enc, 64, seed=3)
    H = h.csr()
    assert not np.any((H @ c.T.astype(np.int64)) % 2)
    assert np.array_equal(c[:, enc.info_pos], u)  # systematic


def test_channel():
    assert math.isclose(awgn_sigma(0.0, 0.5), 1.0)
    assert math.isclose(awgn_sigma(10 * math.log10(2), 0.5), math.sqrt(0.5))
    c = np.zeros((4000, 100), dtype=np.uint8)
    c[::2] = 1
    y = bpsk_awgn(c, 4.0, 0.5, seed=1)
    sig = awgn_sigma(4.0, 0.5)
    s = 1.0 - 2.0 * c
    err = y - s
    assert abs(err.std() - sig) < 0.01 and abs(err.mean()) < 0.01
    assert np.array_equal(y, bpsk_awgn(c, 4.0, 0.5, seed=1))
    assert not np.array_equal(y, bpsk_awgn(c, 4.0, 0.5, seed=2))
