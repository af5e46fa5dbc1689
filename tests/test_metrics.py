"""Retrieval metrics of the synthetic sweeps, pinned by hand-worked lists."""
import numpy as np
import pytest

from paper_2012_07620_gb300 import metrics


def test_hand_worked_average_precision():
    # gallery labels: items 0..5; query label 1 matches items 1, 3, 5
    yg = np.array([0, 1, 2, 1, -1, 1])
    yq = np.array([1, 2])
    ranked = np.array([[3, 0, 1, 4, 2, 5],    # matches at ranks 1, 3, 6: AP = (1/1 + 2/3 + 3/6) / 3
                       [0, 1, 3, 4, 5, 2]])   # one match (item 2) at rank 6: AP = 1/6
    m = metrics.retrieval_metrics(ranked, yq, yg, ks=(1, 5))
    ap0 = (1.0 + 2.0 / 3.0 + 0.5) / 3.0
    assert m["mAP"] == pytest.approx((ap0 + 1.0 / 6.0) / 2.0)
    assert m["R1"] == pytest.approx(0.5)
    assert m["R5"] == pytest.approx(0.5)


def test_truncated_list_counts_missing_matches_as_zero():
    yg = np.array([1, 1, 0, 0])
    yq = np.array([1])
    full = metrics.retrieval_metrics(np.array([[0, 2, 3, 1]]), yq, yg)
    trunc = metrics.retrieval_metrics(np.array([[0, 2]]), yq, yg)
    assert full["mAP"] == pytest.approx((1.0 + 2.0 / 4.0) / 2.0)
    assert trunc["mAP"] == pytest.approx(0.5)


def test_perfect_ranking_and_unmatched_queries():
    yg = np.array([2, 2, 3, -1])
    yq = np.array([2, 7])  # the second query has no match: left out
    m = metrics.retrieval_metrics(np.array([[0, 1, 2, 3], [3, 2, 1, 0]]), yq, yg)
    assert m["mAP"] == 1.0 and m["R1"] == 1.0 and m["queries"] == 1


def test_k1_rule_of_eq15():
    assert metrics.k1_from_classes(23100, 1501) == 15
    assert metrics.k1_from_classes(10, 20) == 1
    with pytest.raises(ValueError):
        metrics.k1_from_classes(10, 0)
