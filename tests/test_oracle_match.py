"""Pins of the oracle's detection-quality count (Eqs. 2 and 3): exact
fractions by brute force in Python, hand cases, and the strict inequalities
(IoU equal to the threshold is neither a true nor a false detection)."""
from fractions import Fraction

import numpy as np

import oracle


def _iou(a, b):
    t = min(a[1], b[1]) - max(a[0], b[0]) + 1
    f = min(a[3], b[3]) - max(a[2], b[2]) + 1
    inter = t * f if t > 0 and f > 0 else 0
    area = lambda x: (x[1] - x[0] + 1) * (x[3] - x[2] + 1)
    return Fraction(inter, area(a) + area(b) - inter)


def _brute(gt, det, thetas):
    gbest = [max((_iou(g, d) for d in det), default=Fraction(0)) for g in gt]
    dbest = [max((_iou(d, g) for g in gt), default=Fraction(0)) for d in det]
    return ([sum(1 for v in gbest if v > th) for th in thetas],
            [sum(1 for v in dbest if v < th) for th in thetas], gbest, dbest)


def _rand_boxes(rng, n, T=60, F=80):
    t0 = rng.integers(0, T, n)
    f0 = rng.integers(0, F, n)
    return np.stack([t0, t0 + rng.integers(0, 12, n), f0, f0 + rng.integers(0, 15, n)], 1)


def test_match_equals_exact_fractions_on_random_sets():
    rng = np.random.default_rng(4)
    thetas = [Fraction(1, 10), Fraction(1, 4), Fraction(1, 3), Fraction(1, 2), Fraction(3, 4)]
    for _ in range(20):
        gt = _rand_boxes(rng, int(rng.integers(0, 25)))
        det = _rand_boxes(rng, int(rng.integers(0, 25)))
        r = oracle.match(gt, det, [float(t) for t in thetas])
        nt, nf, gb, db = _brute(gt.tolist(), det.tolist(), thetas)
        assert r["n_t"].tolist() == nt and r["n_f"].tolist() == nf
        assert [Fraction(int(i), int(u)) for i, u in r["gt_best"]] == gb
        assert [Fraction(int(i), int(u)) for i, u in r["det_best"]] == db


def test_hand_cases_and_ties():
    a = [0, 9, 0, 9]                       # 100 cells
    half = [0, 4, 0, 9]                    # 50 cells inside a: IoU 1/2
    far = [50, 55, 50, 55]
    r = oracle.match(np.array([a]), np.array([a, half, far]), [0.5, 0.49, 0.99])
    assert r["gt_best"].tolist() == [[100, 100]]
    assert r["det_best"].tolist() == [[100, 100], [50, 100], [0, 1]]
    # at theta = 1/2 the half box is neither true nor false; below it, true
    assert r["n_t"].tolist() == [1, 1, 1]
    assert r["n_f"].tolist() == [1, 1, 2]
    # empty sets
    e = oracle.match(np.zeros((0, 4)), np.array([a]), [0.5])
    assert e["n_t"].tolist() == [0] and e["n_f"].tolist() == [1]
    e = oracle.match(np.array([a]), np.zeros((0, 4)), [0.5])
    assert e["n_t"].tolist() == [0] and e["n_f"].tolist() == [0]
