"""The delay formulas of Sec. IV against the paper's worked example."""
from paper_1206_3362_gb300 import delay_model as dm


def test_eg255_worked_example():
    """Sec. IV: EG(255,175), 16 parallel metric units (8 comparators in the
    first stage): the metrics take 16 clocks, FWBF's bit choice 20 clocks per
    iteration, lambda-largest selection 24 lambda clocks."""
    assert dm.sweep_clocks(255, 16) == 16
    assert dm.fwbf_choice_clocks(255, 16) == 20
    for lam in (1, 2, 10):
        assert dm.lambda_choice_clocks(255, 16, lam) == 24 * lam


def test_fig1_network():
    """Fig. 1: 2q = 8 values (q = 4 first-stage comparators) give their
    maximum after log2(8) = 3 clocks; one block of 8 bits is 1 + 3 clocks."""
    assert dm.fwbf_choice_clocks(8, 8) == 4
    assert dm.lambda_choice_clocks(8, 8, 1) == 4


def test_fwbf_never_slower_than_one_global_maximum():
    for N in (255, 504, 1023, 4095, 16384):
        for two_q in (2, 8, 16, 64):
            assert dm.fwbf_choice_clocks(N, two_q) <= dm.lambda_choice_clocks(N, two_q, 1)
