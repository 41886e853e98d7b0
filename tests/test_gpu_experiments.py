"""Sec. V experiments on the GPU: the averaged iterations of Tab. 1 (FWBF,
K_max = 10, EG(1023,781)) reproduced within a statistical band, and the
K_max = 5 / 10 comparison on EG(255,175)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


def test_tab1_fwbf_rows(built):
    """Counting Step-1 evaluations (flip passes + 1), FWBF with alpha = 1.5
    matches both FWBF rows of Tab. 1 within 6 % at 3.5 - 4.5 dB (the paper
    states neither alpha nor its seeds, so only a band is checked)."""
    from paper_1206_3362_gb300 import experiments

    res = experiments.tab1(frames=1 << 15)
    paper = experiments.TAB1
    for i, eb in enumerate(paper["ebn0_db"]):
        if eb < 3.5:
            continue
        row = res["rows"][f"{eb}dB"]
        for key, col in (("fwbf_p31", "fwbf_p31"), ("fwbf_p93", "fwbf_p93")):
            got = row[key]["avg_step1"]
            assert abs(got - paper[col][i]) / paper[col][i] < 0.06, (eb, key, got)
        # the paper's observation: the longer block needs more iterations
        assert row["fwbf_p93"]["avg_step1"] > row["fwbf_p31"]["avg_step1"]


def test_eg255_kmax5_vs_10(built):
    """With 16-bit blocks, 5 and 10 iterations give close error rates on
    EG(255,175) (Sec. V: 'not distinct'); 10 is never worse."""
    from paper_1206_3362_gb300 import experiments

    res = experiments.eg255(frames=1 << 16, ebn0=(4.0, 4.5))
    for row in res["rows"].values():
        assert row["p16_kmax10"]["fer"] <= row["p16_kmax5"]["fer"]
        assert row["p16_kmax5"]["ber"] <= 2.0 * row["p16_kmax10"]["ber"] + 1e-6


def test_scale4_small(built):
    """Learned + batched at scale, on 512 frames per code and point: the
    rate-0.94 column-weight-4 QC code is beyond bit flipping at 4 dB in both
    arms, EG(4095,3367) decodes at 5.5 dB in both."""
    from paper_1206_3362_gb300 import experiments

    out = experiments.scale4(frames=8 * 512, reps=1)
    assert out["frames_per_job"] == 512 and len(out["jobs"]) == 8
    assert out["plain"]["launches"] == 8 and out["learned_batched"]["launches"] == 1
    rows = {(r["code"], r["ebn0_db"]): r for r in out["jobs"]}
    for arm in ("plain", "batched"):
        assert rows[("qc16384", 4.0)][arm]["fer"] >= 0.9
        assert rows[("eg4095", 5.5)][arm]["fer"] <= 0.01
        for r in out["jobs"]:
            assert 0.0 <= r[arm]["ber"] <= r[arm]["fer"] <= 1.0
