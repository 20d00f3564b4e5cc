"""Map-quality metrics (paper Sec. V: IoU of labels at labelled 3D points,
Sec. V-C: AUC of the occupancy probability) against hand-computed values,
all-pairs counting and the geometry of the free-space probes.  CPU only."""
import numpy as np
import pytest

from paper_1909_04631_gb300 import evaluate as ev


def test_confusion_and_iou_by_hand():
    gt = np.array([0] * 6 + [1] * 6 + [2] * 4)
    pred = np.array([0, 0, 0, 0, 0, 1, 0, 0, 1, 1, 1, 2, 2, 2, 2, 2])
    conf = ev.confusion(pred, gt, 3)
    np.testing.assert_array_equal(conf, [[5, 1, 0], [2, 3, 1], [0, 0, 4]])
    # TP / (TP + FP + FN): 5/(5+2+1), 3/(3+1+3), 4/(4+1+0)
    np.testing.assert_allclose(ev.iou(conf), [5 / 8, 3 / 7, 4 / 5], rtol=1e-15)
    assert np.isnan(ev.iou(np.zeros((2, 2))))[0]


def test_auc_equals_pair_counting_with_ties():
    rng = np.random.default_rng(3)
    s = rng.integers(0, 6, size=300).astype(np.float64)  # many ties
    pos = rng.random(300) < 0.4
    sp, sn = s[pos][:, None], s[~pos][None, :]
    brute = ((sp > sn).sum() + 0.5 * (sp == sn).sum()) / (sp.size * sn.size)
    assert ev.roc_auc(s, pos) == pytest.approx(brute, abs=1e-12)


def test_auc_limits():
    pos = np.array([True] * 5 + [False] * 7)
    assert ev.roc_auc(np.r_[np.arange(5) + 10.0, np.arange(7)], pos) == 1.0
    assert ev.roc_auc(np.r_[np.arange(5), np.arange(7) + 10.0], pos) == 0.0
    assert ev.roc_auc(np.ones(12), pos) == 0.5
    assert np.isnan(ev.roc_auc(np.ones(3), np.ones(3, bool)))


def test_auc_matches_scikit_learn():
    metrics = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(4)
    s = np.round(rng.normal(size=2000), 2)
    pos = rng.random(2000) < s.clip(-2, 2) / 4 + 0.5
    assert ev.roc_auc(s, pos) == pytest.approx(metrics.roc_auc_score(pos, s), abs=1e-12)


def test_beam_probes_lie_between_free_samples():
    T = np.eye(4)
    T[:3, 3] = [0.02, 0.05, 0.05]
    q = ev.beam_probes(np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.1]], np.float32), T, 0.3, stride=1)
    # beam 0: r = 1, probes at 0.85, 0.55, 0.25; beam 1: r = 0.1 < step / 2, none
    np.testing.assert_allclose(q, [[0.87, 0.05, 0.05], [0.57, 0.05, 0.05], [0.27, 0.05, 0.05]], atol=1e-6)
    q2 = ev.beam_probes(np.array([[0.0, 0.0, 0.2]], np.float32), T, 0.3, stride=1)
    np.testing.assert_allclose(q2, [[0.02, 0.05, 0.10]], atol=1e-6)


def test_map_quality_of_perfect_and_blind_maps():
    rng = np.random.default_rng(5)
    T = np.eye(4)
    scans = [dict(points=rng.uniform(-5, 5, size=(200, 3)).astype(np.float32),
                  clean_labels=rng.integers(1, 4, size=200).astype(np.int32), pose=T) for _ in range(2)]
    calls = []

    def perfect(xyz):  # hits first, then the probes of the same scan
        k = len(calls)
        calls.append(len(xyz))
        if k % 2 == 0:
            return dict(label=scans[k // 2]["clean_labels"], p_occ=np.ones(len(xyz)))
        return dict(label=np.zeros(len(xyz), np.int32), p_occ=np.zeros(len(xyz)))

    q = ev.map_quality(perfect, scans, 3, step=0.3, stride=4)
    assert q["miou"] == 1.0 and q["auc"] == 1.0 and q["hits"] == 400
    assert q["free_probes"] == calls[1] + calls[3] > 0

    def blind(xyz):  # the prior everywhere: label 0 (ties to the lowest class), p_occ K/(K+1)
        return dict(label=np.zeros(len(xyz), np.int32), p_occ=np.full(len(xyz), 0.75))

    b = ev.map_quality(blind, scans, 3, step=0.3, stride=4)
    assert b["miou"] == 0.0 and b["auc"] == 0.5
