"""Host logic of the learned slice-count policy (no GPU): the tensor work of the check-driven
escalation, the threshold choice by expected work, and the selector_eval summary the benchmark
reports."""
import numpy as np

from paper_2503_22875_gb300 import selector

P = lambda s: s * (s + 1) // 2  # noqa: E731  slice products of one pass


def test_escalation_work_closed_forms():
    fb = 13
    # s1 >= s_min: one pass
    prod, passes = selector.escalation_work([9, 12], [9, 5], fb)
    assert list(prod) == [P(9), P(12)] and list(passes) == [1, 1]
    # short by one or two: the pass at s1 + 2 suffices
    prod, passes = selector.escalation_work([7, 8], [8, 10], fb)
    assert list(prod) == [P(7) + P(9), P(8) + P(10)] and list(passes) == [2, 2]
    # short by three or more: s1, s1 + 2, then the fallback
    prod, passes = selector.escalation_work([6], [9], fb)
    assert list(prod) == [P(6) + P(8) + P(13)] and list(passes) == [3]
    # s1 + 2 capped at the fallback; no third pass when the second is at the fallback
    prod, passes = selector.escalation_work([12, 12], [13, 16], fb)
    assert list(prod) == [P(12) + P(13)] * 2 and list(passes) == [2, 2]
    # counts at or above the fallback are never escalated
    prod, passes = selector.escalation_work([13, 14], [16, 16], fb)
    assert list(prod) == [P(13), P(14)] and list(passes) == [1, 1]


def test_choose_threshold_minimises_expected_work():
    # two GEMMs; class probabilities over s = 2..12.  GEMM 0 needs 8 and is sure of it; GEMM 1
    # needs 10 but its model spreads 60% on 8 and 40% on 10.
    probs = np.zeros((2, 11))
    probs[0, 8 - 2] = 1.0
    probs[1, 8 - 2], probs[1, 10 - 2] = 0.6, 0.4
    s_min = np.array([8, 10])
    work = np.array([1.0, 1.0])
    best, table = selector.choose_threshold(probs, s_min, work, 13, grid=[0.5, 0.9])
    # thr 0.5: (8, 8) -> GEMM 1 re-runs at 10: 36 + 36 + 55; thr 0.9: (8, 10): 36 + 55
    assert table[0.5]["cost"] == P(8) + P(8) + P(10)
    assert table[0.9]["cost"] == P(8) + P(10)
    assert best == 0.9 and table[0.5]["rerun_frac"] == 0.5 and table[0.9]["rerun_frac"] == 0.0


def test_selector_eval_arithmetic():
    sel = [7, 8, 9, 10, 12, 6]
    smin = [7, 9, 9, 8, 9, 6]
    work = [1, 2, 3, 4, 5, 6]
    e = selector.selector_eval(sel, smin, work)
    assert e["calls"] == 6
    assert e["exact"] == 3 / 6 and e["over"] == 2 / 6 and e["under"] == 1 / 6
    assert e["mean_excess_slices_when_over"] == (2 + 3) / 2
    assert e["mean_shortfall_when_under"] == 1.0
    assert e["mean_selected"] == np.mean(sel) and e["mean_minimum"] == np.mean(smin)
    assert e["work_weighted"] == {"exact": 10 / 21, "over": 9 / 21, "under": 2 / 21}
    # all exact: no excess, no shortfall
    e = selector.selector_eval([5, 6], [5, 6])
    assert e["exact"] == 1.0 and e["mean_excess_slices_when_over"] == 0.0 and "work_weighted" not in e
