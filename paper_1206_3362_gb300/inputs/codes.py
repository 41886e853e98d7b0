"""Seeded parity-check matrix builders for the LDPC codes the decoder is run on.

This module builds inputs only: it holds no step of the decoding method.  Every
builder returns a :class:`ParityCheck` whose ``rows``/``cols`` are the COO
coordinates of the ones of H (the form ``fwbf_code_create`` takes).

Codes:

* ``eg2_cyclic(s)``: type-I two-dimensional Euclidean-geometry code EG(2, 2^s).
  The paper decodes the EG (255,175) and EG (1023,781) codes (s = 4, 5; Sec. V);
  s = 6 gives (4095,3367).  H is the circulant incidence matrix of the lines of
  EG(2, 2^s) that miss the origin against its non-origin points, so both row and
  column weight are 2^s and any two lines meet in at most one point (the RC
  constraint of Sec. II).
* ``random_regular(N, dv, dc, seed)``: (dv, dc)-regular code from a random socket
  permutation with every double edge and 4-cycle removed by random edge swaps.
* ``quasi_cyclic(Z, shifts)`` / ``random_qc(...)``: H made of Z x Z blocks,
  each zero or a sum of circulant permutation matrices.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class ParityCheck:
    """Binary M x N parity-check matrix H in COO form (one entry per 1)."""

    N: int
    M: int
    rows: np.ndarray  # int32 [nnz] check index m of each one
    cols: np.ndarray  # int32 [nnz] bit index n of each one
    name: str = ""
    circulant: int = 1  # Z when H is known to be built from Z x Z circulants

    @property
    def nnz(self) -> int:
        return int(self.rows.size)

    def dense(self) -> np.ndarray:
        h = np.zeros((self.M, self.N), dtype=np.uint8)
        h[self.rows, self.cols] = 1
        return h

    def csr(self) -> sp.csr_matrix:
        data = np.ones(self.nnz, dtype=np.int32)
        return sp.csr_matrix((data, (self.rows, self.cols)), shape=(self.M, self.N))

    def row_weights(self) -> np.ndarray:
        return np.bincount(self.rows, minlength=self.M)

    def col_weights(self) -> np.ndarray:
        return np.bincount(self.cols, minlength=self.N)

    def max_row_overlap(self) -> int:
        """Largest number of columns two distinct rows share (RC constraint: <= 1)."""
        h = self.csr()
        g = (h @ h.T).tocoo()
        off = g.row != g.col
        return int(g.data[off].max()) if off.any() else 0

    def max_col_overlap(self) -> int:
        h = self.csr()
        g = (h.T @ h).tocoo()
        off = g.row != g.col
        return int(g.data[off].max()) if off.any() else 0

    def has_duplicates(self) -> bool:
        key = self.rows.astype(np.int64) * self.N + self.cols
        return np.unique(key).size != key.size


# ---------------------------------------------------------------------------
# GF(2^m) arithmetic for the Euclidean-geometry construction
# ---------------------------------------------------------------------------

def _poly_x_order(poly: int, m: int) -> int:
    """Multiplicative order of x modulo the degree-m binary polynomial ``poly``
    (0 when x is not invertible / the powers never return to 1 within 2^m-1)."""
    top = 1 << m
    v = 1
    for k in range(1, top):
        v <<= 1
        if v & top:
            v ^= poly
        if v == 1:
            return k
    return 0


def primitive_polynomial(m: int) -> int:
    """Smallest binary polynomial of degree m whose root x has order 2^m - 1,
    i.e. a primitive polynomial, found by search (no stored table)."""
    target = (1 << m) - 1
    for poly in range((1 << m) | 1, 1 << (m + 1), 2):
        if _poly_x_order(poly, m) == target:
            return poly
    raise ValueError(f"no primitive polynomial of degree {m}")


def gf_tables(m: int):
    """exp / log tables of GF(2^m) for the primitive element alpha = x."""
    poly = primitive_polynomial(m)
    q = 1 << m
    exp = np.zeros(2 * q, dtype=np.int64)
    log = np.full(q, -1, dtype=np.int64)
    v = 1
    for k in range(q - 1):
        exp[k] = v
        log[v] = k
        v <<= 1
        if v & q:
            v ^= poly
    exp[q - 1: 2 * (q - 1)] = exp[: q - 1]
    return exp, log


def eg2_offsets(s: int) -> np.ndarray:
    """Exponent set D of one line of EG(2, 2^s) that misses the origin.

    The points of EG(2, 2^s) are the elements of GF(2^(2s)); the non-origin ones
    are alpha^0 .. alpha^(n-1), n = 2^(2s) - 1.  The line {1 + beta*alpha : beta in
    GF(2^s)} does not contain 0 (alpha is not in the subfield) and has 2^s points.
    Multiplying it by alpha^m gives every other line that misses the origin, so
    H[m][n] = 1 iff (n - m) mod n_pts is in D.
    """
    m = 2 * s
    exp, log = gf_tables(m)
    n_pts = (1 << m) - 1
    step = (1 << s) + 1  # alpha^(k*step) for k = 0..2^s-2 is GF(2^s)*
    alpha = int(exp[1])
    pts = [1]  # beta = 0
    for k in range(0, (1 << s) - 1):
        beta = int(exp[(k * step) % n_pts])
        # beta * alpha in GF(2^m) through the log tables
        prod = int(exp[(log[beta] + log[alpha]) % n_pts])
        pts.append(1 ^ prod)
    d = np.array(sorted(int(log[p]) for p in pts), dtype=np.int64)
    if np.unique(d).size != (1 << s):
        raise AssertionError("line points are not distinct")
    return d


def eg2_cyclic(s: int) -> ParityCheck:
    """Type-I cyclic EG(2, 2^s) LDPC code: N = M = 4^s - 1, weights 2^s."""
    d = eg2_offsets(s)
    n = (1 << (2 * s)) - 1
    m_idx = np.repeat(np.arange(n, dtype=np.int64), d.size)
    n_idx = (m_idx + np.tile(d, n)) % n
    return ParityCheck(N=n, M=n, rows=m_idx.astype(np.int32), cols=n_idx.astype(np.int32),
                       name=f"EG(2,2^{s})", circulant=n)


# ---------------------------------------------------------------------------
# Random regular codes without 4-cycles
# ---------------------------------------------------------------------------

def _bad_edges(rows: np.ndarray, cols: np.ndarray, M: int, N: int) -> np.ndarray:
    """Indices of edges that are duplicated or lie on a 4-cycle."""
    key = rows.astype(np.int64) * N + cols
    order = np.argsort(key, kind="stable")
    dup = np.zeros(rows.size, dtype=bool)
    same = key[order][1:] == key[order][:-1]
    dup[order[1:][same]] = True
    data = np.ones(rows.size, dtype=np.int32)
    h = sp.csr_matrix((data, (rows, cols)), shape=(M, N))
    h.data[:] = 1
    g = (h @ h.T).tocoo()
    sel = (g.row < g.col) & (g.data >= 2)
    bad = dup.copy()
    if sel.any():
        # mark one edge of every offending check pair: an edge of the first
        # check that lands on a column shared with the second
        hcsr = h.tocsr()
        for m1, m2 in zip(g.row[sel], g.col[sel]):
            shared = np.intersect1d(hcsr.indices[hcsr.indptr[m1]:hcsr.indptr[m1 + 1]],
                                    hcsr.indices[hcsr.indptr[m2]:hcsr.indptr[m2 + 1]])
            e = np.nonzero((rows == m1) & (cols == shared[0]))[0]
            bad[e[0]] = True
    return np.nonzero(bad)[0]


def random_regular(N: int, dv: int, dc: int, seed: int, max_rounds: int = 10000) -> ParityCheck:
    """(dv, dc)-regular H from a seeded random socket permutation; double edges
    and 4-cycles are removed by swapping the check ends of random edge pairs."""
    if (N * dv) % dc:
        raise ValueError("N*dv must be a multiple of dc")
    M = N * dv // dc
    rng = np.random.Generator(np.random.Philox(seed))
    cols = np.repeat(np.arange(N, dtype=np.int32), dv)
    rows = np.repeat(np.arange(M, dtype=np.int32), dc)
    rows = rows[rng.permutation(rows.size)]
    for _ in range(max_rounds):
        bad = _bad_edges(rows, cols, M, N)
        if bad.size == 0:
            return ParityCheck(N=N, M=M, rows=rows.copy(), cols=cols.copy(),
                               name=f"random({dv},{dc}) N={N} seed={seed}")
        partners = rng.integers(0, rows.size, size=bad.size)
        for e, f in zip(bad, partners):
            rows[e], rows[f] = rows[f], rows[e]
    raise RuntimeError("4-cycle removal did not converge")


# ---------------------------------------------------------------------------
# Quasi-cyclic codes
# ---------------------------------------------------------------------------

def quasi_cyclic(Z: int, shifts) -> ParityCheck:
    """H from a base matrix of circulant shift sets.

    ``shifts[r][c]`` is a (possibly empty) list of shifts t; block (r, c) is the
    sum of the Z x Z circulant permutations P^t with ones at (i, (i + t) mod Z).
    """
    mb = len(shifts)
    nb = len(shifts[0])
    rows, cols = [], []
    i = np.arange(Z, dtype=np.int64)
    for r in range(mb):
        for c in range(nb):
            for t in shifts[r][c]:
                rows.append(r * Z + i)
                cols.append(c * Z + (i + int(t)) % Z)
    return ParityCheck(N=nb * Z, M=mb * Z, rows=np.concatenate(rows).astype(np.int32),
                       cols=np.concatenate(cols).astype(np.int32), circulant=Z)


def random_qc(Z: int, mb: int, nb: int, seed: int, weight: int = 1,
              max_tries: int = 1000) -> ParityCheck:
    """Seeded QC code: mb x nb blocks, each the sum of ``weight`` distinct
    circulant permutations, with no 4-cycles.

    Shifts are drawn one block column at a time; a column is redrawn while the
    matrix built so far has two rows sharing more than one column (a 4-cycle).
    """
    rng = np.random.Generator(np.random.Philox(seed))
    shifts = [[[] for _ in range(nb)] for _ in range(mb)]
    for c in range(nb):
        for _ in range(max_tries):
            for r in range(mb):
                shifts[r][c] = sorted(rng.choice(Z, size=weight, replace=False).tolist())
            part = quasi_cyclic(Z, [row[: c + 1] for row in shifts])
            if part.max_row_overlap() <= 1:
                break
        else:
            raise RuntimeError("could not place circulant shifts without 4-cycles")
    h = quasi_cyclic(Z, shifts)
    h.name = f"QC Z={Z} {mb}x{nb} w={weight} seed={seed}"
    return h
