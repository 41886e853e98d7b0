"""Host logic of bench.py (no GPU): the clock record kept beside each number."""
import datetime

import bench

ROWS = """2026/12/04 04:32:22.900, 0, 1980, 2070, 610.2, 0x0, Not Active, Not Active, Not Active, Not Active
2026/12/04 04:32:23.000, 0, 2070, 2070, 905.1, 0x0, Not Active, Not Active, Not Active, Not Active
2026/12/04 04:32:23.100, 0, 2055, 2070, 1210.7, 0x4, Not Active, Not Active, Not Active, Active
2026/12/04 04:32:23.200, 0, 2070, 2070, 1190.0, 0x0, Not Active, Not Active, Not Active, Not Active
2026/12/04 04:32:23.300, 0, 1500, 2070, 400.0, 0x40, Not Active, Active, Not Active, Not Active
[N/A], 0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active
"""


def _t(s):
    return datetime.datetime.strptime("2026/12/04 04:32:" + s, "%Y/%m/%d %H:%M:%S.%f")


def test_parse_rows():
    rows = bench.ClockSampler.parse(ROWS)
    assert len(rows) == 5  # the row without a clock reading is dropped
    assert rows[0][0] == _t("22.900") and rows[0][1:3] == (1980.0, 2070.0)
    assert rows[2][3] == ["sw_power_cap"] and rows[4][3] == ["hw_thermal_slowdown"]


def test_summary_keeps_the_timed_region():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = _t("22.950"), _t("23.250")
    out = c.summarise(bench.ClockSampler.parse(ROWS))
    assert out["window"] == "timed region" and out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]  # the thermal row lies after the region


def test_summary_says_when_no_sample_is_inside():
    c = bench.ClockSampler(0)
    c.t0, c.t1 = _t("23.310"), _t("23.390")
    out = c.summarise(bench.ClockSampler.parse(ROWS))
    assert out["window"].startswith("whole run") and out["samples"] == 5
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_unparsable_timestamps_fall_back_to_every_row():
    text = ROWS.replace("2026/12/04 04:32:23.100", "Thu Dec  4 04:32:23 2026")
    c = bench.ClockSampler(0)
    c.t0, c.t1 = _t("22.950"), _t("23.250")
    out = c.summarise(bench.ClockSampler.parse(text))
    assert out["samples"] == 2 and out["window"] == "timed region"


class _FakeCode:
    handle = None

    def outputs(self, F, device=None):
        import torch

        return torch.zeros((F, 1), dtype=torch.int32), torch.zeros(F, dtype=torch.int32)


class _FakeDecoder:
    """Frame f's decisions after m passes: a frame that settles at pass j
    (its pass j flips nothing) holds state min(m, j); a frame with a 2-cycle
    from pass j alternates j, j + 1 (never settles)."""

    def __init__(self, settle, cycle):
        self.settle, self.cycle = settle, cycle
        self.handle = None

    def state(self, f, m):
        j = self.settle[f]
        if self.cycle[f]:
            return m if m < j else j + ((m - j) % 2)
        return min(m, j)

    def fwbf_decode(self, handle, q, m, alpha, bits, iters):
        for r in range(q.shape[0]):
            f = int(q[r, 0])
            bits[r, 0] = self.state(f, m)
            iters[r] = -m


def test_executed_passes_counts_the_fixed_point_pass():
    """Converged frames run iters passes; a failing frame that settles after j
    flipping passes runs j + 1 (the last finds no flip); one that never
    settles runs max_iter."""
    import torch

    max_iter = 20
    settle = [3, 7, 0, 5, 19, 4]
    cycle = [False, False, False, True, False, False]
    iters = torch.tensor([3, -max_iter, -max_iter, -max_iter, -max_iter, 2], dtype=torch.int32)
    fake = _FakeDecoder(settle, cycle)
    q = torch.arange(6, dtype=torch.int32).reshape(6, 1)
    bits = torch.tensor([[fake.state(f, max_iter)] for f in range(6)], dtype=torch.int32)
    z0 = torch.tensor([[fake.state(f, 0)] for f in range(6) if iters[f] < 0], dtype=torch.int32)
    got = bench.executed_passes(fake, _FakeCode(), q, bits, iters, max_iter, 1.5, z0=z0)
    assert got.tolist() == [3, 8, 1, max_iter, max_iter, 2]


def test_hard_decisions_packed_like_the_outputs():
    import torch

    q = torch.zeros((2, 40), dtype=torch.int8)
    q[0, [0, 5, 31, 32, 39]] = -3
    q[1, 33] = -127
    z = bench.pack_hard_decisions(q)
    w = [[int(v) & 0xffffffff for v in row] for row in z.tolist()]
    assert w[0] == [(1 << 0) | (1 << 5) | (1 << 31), (1 << 0) | (1 << 7)] and w[1] == [0, 1 << 1]
