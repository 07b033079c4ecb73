"""The P/R/F tool on hand-built cases (section "Results and Discussion" defines
P = TP / (TP + FP), R = TP / (TP + FN), F = 2PR / (P + R))."""
import numpy as np
import pytest

from paper_1804_06304_gb300.evaluate import detection_prf, match_inside


def test_inside_rule_and_one_to_one():
    truth = np.array([[0.0, 0.0], [10.0, 0.0], [20.0, 0.0]])
    radii = np.array([2.0, 2.0, 2.0])
    det = np.array([[0.5, 0.0],      # inside nucleus 0
                    [0.0, 1.0],      # also inside nucleus 0: only one may match
                    [11.9, 0.0],     # inside nucleus 1
                    [22.0, 0.0]])    # on the boundary of nucleus 2: outside (strict)
    assert match_inside(det, truth, radii) == 2
    r = detection_prf(det, truth, radii)
    assert (r["tp"], r["fp"], r["fn"]) == (2, 2, 1)
    assert r["precision"] == pytest.approx(0.5) and r["recall"] == pytest.approx(2 / 3)
    assert r["f"] == pytest.approx(2 * 0.5 * (2 / 3) / (0.5 + 2 / 3))


def test_closest_pairs_first():
    # detection a is inside both nuclei; b only inside nucleus 1: closest-first gives 2 matches
    truth = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    radii = np.array([2.5, 2.5])
    det = np.array([[1.4, 0.0, 0.0], [4.0, 0.0, 0.0]])
    assert match_inside(det, truth, radii) == 2


def test_empty_sets():
    assert detection_prf(np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(0))["f"] == 0.0
    r = detection_prf(np.zeros((0, 3)), np.ones((4, 3)), np.ones(4))
    assert (r["tp"], r["fn"], r["recall"]) == (0, 4, 0.0)


def test_perfect_detection_of_synthetic_nuclei():
    from paper_1804_06304_gb300 import synth
    s = synth.small_3d(0)
    r = detection_prf(s.centres + 0.3, s.centres, s.radii)
    assert r["precision"] == 1.0 and r["recall"] == 1.0 and r["f"] == 1.0
