"""Host logic of the autotuner (no GPU): the FER qualification rule and the
result cache."""
import json
import os

from paper_1206_3362_gb300 import autotune


def _r(p, alpha, fe, be, ms):
    return {"p": p, "alpha": alpha, "frame_errors": fe, "bit_errors": be, "ms": ms}


def test_fastest_setting_that_is_no_worse_wins():
    ref = _r(31, 1.5, 10, 200, 5.0)
    results = [
        _r(1, 1.0, 9, 150, 2.0),     # better on both counts but slower than the winner
        _r(8, 2.0, 10, 200, 1.5),    # equal errors, fastest qualified
        _r(16, 2.0, 11, 100, 1.0),   # one more frame error: excluded despite being fastest
        _r(4, 1.0, 8, 201, 1.2),     # one more bit error: excluded
        ref,
    ]
    assert autotune.select_fastest_qualified(results, ref) is results[1]


def test_reference_always_qualifies():
    ref = _r(31, 1.5, 3, 40, 9.0)
    results = [_r(8, 2.0, 4, 10, 1.0), _r(16, 1.0, 2, 41, 2.0), ref]
    assert autotune.select_fastest_qualified(results, ref) is ref


def test_bit_errors_decide_when_every_frame_fails():
    """On a code beyond bit flipping's reach every setting fails every frame;
    only settings with no more bit errors than the reference are admitted."""
    ref = _r(32, 1.5, 100, 5000, 3.0)
    results = [_r(8, 2.0, 100, 5200, 1.0), _r(16, 1.5, 100, 4900, 2.5), ref]
    assert autotune.select_fastest_qualified(results, ref) is results[1]


def test_ties_in_time_keep_the_earlier_setting():
    ref = _r(31, 1.5, 5, 50, 2.0)
    results = [_r(8, 1.0, 5, 50, 2.0), _r(8, 2.0, 5, 50, 2.0), ref]
    assert autotune.select_fastest_qualified(results, ref) is results[0]


def test_cache_round_trip(tmp_path):
    path = os.path.join(tmp_path, "sub", "autotune.json")
    c = autotune.Cache(path)
    assert c.get("k") is None
    c.put("k", {"choice": {"p": 8, "alpha": 2.0}})
    with open(path) as f:
        assert json.load(f) == {"k": {"choice": {"p": 8, "alpha": 2.0}}}
    assert autotune.Cache(path).get("k") == {"choice": {"p": 8, "alpha": 2.0}}
    assert not [n for n in os.listdir(os.path.dirname(path)) if ".tmp" in n]


def test_cache_ignores_a_damaged_file(tmp_path):
    path = os.path.join(tmp_path, "autotune.json")
    with open(path, "w") as f:
        f.write("{not json")
    assert autotune.Cache(path).get("k") is None


def _g(gate, fe, ms):
    return {"gate_dv": gate, "frame_errors": fe, "bit_errors": 10 * fe, "ms": ms}


def test_gate_keeps_half_the_network_gain():
    """Ungated network 100 frame errors, plain FWBF 300: gates with at most
    200 qualify; the fastest of them wins, a faster gate with 201 does not."""
    plain = {"frame_errors": 300, "bit_errors": 3000, "ms": 10.0}
    results = [_g(0, 100, 12.0), _g(6, 110, 11.5), _g(12, 200, 10.8), _g(16, 201, 10.1)]
    assert autotune.select_gate(results, plain) is results[2]


def test_ungated_network_always_qualifies():
    plain = {"frame_errors": 90, "bit_errors": 900, "ms": 10.0}
    results = [_g(0, 100, 12.0), _g(6, 96, 11.0), _g(12, 96, 10.5)]
    assert autotune.select_gate(results, plain) is results[0]


def test_gate_near_tie_goes_to_fewer_errors():
    """Qualifying gates within 1 % of the fastest time (the EG(4095)
    calibration at 4 dB: every gate within 0.7 %) are a tie decided by frame
    errors, then bit errors, then time; a gate 1.5 % slower is not in it."""
    plain = {"frame_errors": 8556, "bit_errors": 673673, "ms": 9.9}
    results = [_g(0, 5029, 11.10), _g(6, 5029, 11.05), _g(10, 5035, 11.03), _g(12, 5053, 11.028),
               _g(14, 5073, 11.04), _g(16, 5101, 11.05)]
    assert autotune.select_gate(results, plain) is results[1]
    results = [_g(0, 100, 10.20), _g(6, 140, 10.0), _g(12, 150, 10.05)]
    plain = {"frame_errors": 300, "bit_errors": 3000, "ms": 9.0}
    assert autotune.select_gate(results, plain) is results[1]
