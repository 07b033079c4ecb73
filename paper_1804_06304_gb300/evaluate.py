"""Detection quality against synthetic ground truth: precision, recall and
F-measure as the paper defines them (section "Results and Discussion": P = TP /
(TP + FP), R = TP / (TP + FN), F = 2 P R / (P + R)).

The paper labels its contours cell / non-cell with a KNN classifier on annotated
data; here the synthetic volumes carry their nuclei, so a detected cell is a true
positive when its centre lies inside a ground-truth nucleus (distance below the
nucleus radius), each nucleus matching at most one detection, closest pairs first.
Host-side evaluation only; it takes no part in the evolution.
"""
from __future__ import annotations

import numpy as np


def match_inside(det: np.ndarray, truth: np.ndarray, radius: np.ndarray) -> int:
    """Number of one-to-one pairs (detection, nucleus) with the detection's centre
    inside the nucleus, formed closest first."""
    if len(det) == 0 or len(truth) == 0:
        return 0
    det = np.asarray(det, dtype=np.float64).reshape(len(det), -1)
    truth = np.asarray(truth, dtype=np.float64).reshape(len(truth), -1)
    radius = np.asarray(radius, dtype=np.float64).reshape(-1)
    from scipy.spatial import cKDTree
    tree = cKDTree(truth)
    rmax = float(radius.max())
    pairs = []
    for i, near in enumerate(tree.query_ball_point(det, rmax)):
        for j in near:
            d = float(np.linalg.norm(det[i] - truth[j]))
            if d < radius[j]:
                pairs.append((d, i, j))
    pairs.sort()
    used_d, used_t, m = set(), set(), 0
    for _, i, j in pairs:
        if i not in used_d and j not in used_t:
            used_d.add(i)
            used_t.add(j)
            m += 1
    return m


def detection_prf(det_centres, truth_centres, truth_radii) -> dict:
    """Precision, recall and F-measure of detected centres against nuclei (physical
    coordinates, one row per point, same number of columns)."""
    n_det, n_truth = len(det_centres), len(truth_centres)
    tp = match_inside(det_centres, truth_centres, truth_radii)
    p = tp / n_det if n_det else 0.0
    r = tp / n_truth if n_truth else 0.0
    f = 2 * p * r / (p + r) if p + r > 0 else 0.0
    return {"tp": tp, "fp": n_det - tp, "fn": n_truth - tp, "precision": p, "recall": r, "f": f}
