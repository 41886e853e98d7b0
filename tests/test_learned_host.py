"""Host logic of the learned-schedule pipeline (no GPU): the greedy per-pass
labelling with the decoder replaced by the oracle, the Wilson interval and the
fixed-point alpha."""
import math

import numpy as np
import pytest

import oracle
from paper_1206_3362_gb300 import learned
from paper_1206_3362_gb300.inputs import Encoder, bpsk_awgn, make_code, random_codewords

torch = pytest.importorskip("torch")


def test_alpha_q_rounds_half_to_even():
    assert learned.alpha_q(1.5) == 384
    assert learned.alpha_q(0.5 / 256) == 0
    assert learned.alpha_q(1.5 / 256) == 2
    assert learned.alpha_q(2.5 / 256) == 2


def test_wilson_interval():
    assert learned.wilson(0, 0) == (0.0, 1.0)
    z = 1.96
    lo, hi = learned.wilson(0, 100)
    assert lo == 0.0 and math.isclose(hi, z * z / (100 + z * z), rel_tol=1e-12)
    for k, n in ((3, 50), (17, 40), (99, 100)):
        lo, hi = learned.wilson(k, n)
        assert lo <= k / n <= hi
        lo2, hi2 = learned.wilson(n - k, n)
        assert math.isclose(lo, 1 - hi2, abs_tol=1e-12) and math.isclose(hi, 1 - lo2, abs_tol=1e-12)


class _OracleCode:
    """Stands in for a code handle: outputs on the CPU, decoding by the oracle."""

    def __init__(self, h, p):
        self.h, self.p, self.handle = h, p, object()
        self.words = (h.N + 31) // 32

    def outputs(self, F, device="cpu"):
        return torch.empty((F, self.words), dtype=torch.int32), torch.empty(F, dtype=torch.int32)


def _fake_decode_sched(code):
    def run(handle, q, K, A, T, bits, iters, out_feat=None, stream=None):
        b, it = oracle.fwbf_i8(code.h, code.p, q.numpy(), K, alpha_sched=A.numpy(), theta_sched=T.numpy())
        bits.copy_(torch.from_numpy(b.view(np.int32)))
        iters.copy_(torch.from_numpy(it))
    return run


def _greedy_by_frame(code, q, c, sch):
    """The labelling rule restated frame by frame: at pass k (earlier passes
    at their labels, later ones at the default) take the grid point that
    reaches the transmitted codeword in the fewest passes; the default wins
    ties, then the earlier grid point; a frame stops being labelled once it
    is solved within k + 1 passes or no grid point solves it."""
    K = sch.label_max_iter
    grid = [(learned.alpha_q(a), int(round(t * 256))) for a in sch.grid_alpha for t in sch.grid_theta]
    dflt = (learned.alpha_q(sch.alpha_default), 0)
    F = q.shape[0]
    A = np.full((F, K), dflt[0], dtype=np.int32)
    T = np.zeros((F, K), dtype=np.int32)
    for f in range(F):
        for k in range(sch.k_learn):
            best, best_g = None, None
            for g in [dflt] + [g for g in grid if g != dflt]:
                a, t = A[f:f + 1].copy(), T[f:f + 1].copy()
                a[0, k], t[0, k] = g
                b, it = oracle.fwbf_i8(code.h, code.p, q[f:f + 1], K, alpha_sched=a, theta_sched=t)
                ok = it[0] >= 0 and np.array_equal(oracle.unpack_bits(b, code.h.N)[0], c[f])
                if ok and (best is None or it[0] < best):
                    best, best_g = int(it[0]), g
            if best_g is not None:
                A[f, k], T[f, k] = best_g
            if best is None or best <= k + 1:
                break
    return A, T


def test_label_schedules_follow_the_greedy_rule(monkeypatch):
    h = make_code("eg255")
    enc = Encoder(h)
    _, c = random_codewords(enc, 16, seed=31)
    q = oracle.quantize(bpsk_awgn(c, 2.75, enc.rate, seed=31))
    sch = learned.Schedule(alpha_default=1.5, grid_alpha=(1.0, 1.5, 2.5), grid_theta=(0.0, 4.0), k_learn=3,
                           label_max_iter=20)
    code = _OracleCode(h, 16)
    monkeypatch.setattr(learned.fwbf, "fwbf_decode_sched", _fake_decode_sched(code))
    A, T = learned.label_schedules(code, torch.from_numpy(q), torch.from_numpy(c), sch, chunk=5)
    A2, T2 = _greedy_by_frame(code, q, c, sch)
    assert np.array_equal(A.numpy(), A2) and np.array_equal(T.numpy(), T2)
    assert (A2[:, :sch.k_learn] != 384).any() or (T2[:, :sch.k_learn] != 0).any()
