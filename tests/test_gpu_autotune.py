"""The autotuner only admits FER-qualified settings and picks the fastest of
them; its cache round-trips."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fwbf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    from paper_1206_3362_gb300 import fwbf as mod

    return mod


def test_tune_code_eg1023(fwbf, tmp_path):
    from paper_1206_3362_gb300 import autotune
    from paper_1206_3362_gb300.inputs import Encoder, make_code

    h = make_code("eg1023")
    enc = Encoder(h)
    cache = autotune.Cache(str(tmp_path / "c.json"))
    res = autotune.tuned_code(h, enc, 4.0, p_ref=31, cache=cache, frames=1 << 14,
                              p_candidates=(8, 16, 31), alpha_candidates=(1.5, 2.0))
    ref = res["reference"]
    ch = res["choice"]
    chosen = [r for r in res["candidates"] if r["p"] == ch["p"] and r["alpha"] == ch["alpha"]][0]
    assert chosen["frame_errors"] <= ref["frame_errors"] and chosen["bit_errors"] <= ref["bit_errors"]
    qualified = [r for r in res["candidates"]
                 if r["frame_errors"] <= ref["frame_errors"] and r["bit_errors"] <= ref["bit_errors"]]
    assert chosen["ms"] == min(r["ms"] for r in qualified)
    print("autotune eg1023 4 dB:", res["choice"], "ref", ref, "chosen", chosen)
    again = autotune.Cache(str(tmp_path / "c.json")).get(cache.key(h, 4.0))
    assert again["choice"] == ch
