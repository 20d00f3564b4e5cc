"""Map quality against synthetic ground truth, as the paper's experiments
score a map (Sec. V): the intersection over union TP / (TP + FP + FN) of the
map's labels at labelled 3D points, per class and averaged (SemanticKITTI
evaluation), and the area under the ROC curve of the occupancy probability
(Sec. V-C, Table (occupancy)), with the scans' hits as occupied examples
and points the beams passed through as free ones.

The map is read through the library's read-off (any callable returning the
``label`` and ``p_occ`` arrays of ``Map.query`` for world points); what is
computed here is bookkeeping on the read-off: a confusion matrix and the
rank-sum form of the AUC.
"""
from __future__ import annotations

import numpy as np


def confusion(pred, gt, num_labels: int) -> np.ndarray:
    """[gt, pred] counts of labels in 0..num_labels-1."""
    pred = np.asarray(pred, np.int64).ravel()
    gt = np.asarray(gt, np.int64).ravel()
    return np.bincount(gt * num_labels + pred, minlength=num_labels * num_labels).reshape(num_labels, num_labels)


def iou(conf: np.ndarray) -> np.ndarray:
    """Per class TP / (TP + FP + FN) from a [gt, pred] confusion matrix; NaN
    for a class that is neither in the ground truth nor predicted."""
    conf = np.asarray(conf, np.float64)
    tp = np.diag(conf)
    denom = conf.sum(0) + conf.sum(1) - tp
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(denom > 0, tp / denom, np.nan)


def roc_auc(scores, positive) -> float:
    """Area under the ROC curve: the probability that a random positive scores
    above a random negative, ties counting one half (Mann-Whitney form, from
    the average ranks of tied scores).  NaN without both kinds of example."""
    s = np.asarray(scores, np.float64).ravel()
    pos = np.asarray(positive, bool).ravel()
    n1 = int(pos.sum())
    n0 = len(s) - n1
    if n1 == 0 or n0 == 0:
        return float("nan")
    order = np.argsort(s, kind="mergesort")
    _, start, count = np.unique(s[order], return_index=True, return_counts=True)
    avg = start + (count + 1) / 2.0  # 1-based average rank of each group of equal scores
    ranks = np.empty(len(s))
    ranks[order] = np.repeat(avg, count)
    return float((ranks[pos].sum() - n1 * (n1 + 1) / 2.0) / (n1 * n0))


def to_world(points, pose) -> np.ndarray:
    """Sensor-frame points [n,3] to world coordinates (float32) with a 4x4 pose."""
    T = np.asarray(pose, np.float64).reshape(4, 4)
    return (np.asarray(points, np.float64) @ T[:3, :3].T + T[:3, 3]).astype(np.float32)


def beam_probes(points, pose, step: float, stride: int = 8) -> np.ndarray:
    """Free-space examples: on every stride-th beam, the midpoints between the
    beam's free samples, at ranges r - (j + 1/2) step > 0 for j >= 0 (points
    the beam passed through before its hit).  World frame, float32."""
    T = np.asarray(pose, np.float64).reshape(4, 4)
    p = np.asarray(points, np.float64)[::stride]
    r = np.linalg.norm(p, axis=1)
    keep = r > 0.5 * step
    p, r = p[keep], r[keep]
    n = np.ceil(r / step - 0.5).astype(np.int64)  # j = 0 .. n-1 keep r - (j + 1/2) step > 0
    beam = np.repeat(np.arange(len(p)), n)
    j = np.arange(n.sum()) - np.repeat(np.cumsum(n) - n, n)
    t = r[beam] - (j + 0.5) * step
    q = p[beam] * (t / r[beam])[:, None]
    return (q @ T[:3, :3].T + T[:3, 3]).astype(np.float32)


def map_quality(query, scans, num_classes: int, step: float, stride: int = 8) -> dict:
    """Scores a map on labelled scans: query(xyz) -> dict with "label" and
    "p_occ" (e.g. Map.query); scans: dicts with points (sensor frame),
    clean_labels (ground truth, 1..K) and pose.  Returns the per-class IoU
    over the hits (classes 0..K; a hit read as free counts against its
    class), the mean IoU over the occupied classes present in the ground
    truth, the occupancy AUC (hits against beam_probes) and the counts.
    Occupancy scores are ranked as FP32 values (the read-off's precision),
    so scores that differ only by the rounding of a wider sum tie."""
    K1 = num_classes + 1
    conf = np.zeros((K1, K1), np.int64)
    pos, neg = [], []
    for sc in scans:
        hits = to_world(sc["points"], sc["pose"])
        qh = query(hits)
        conf += confusion(qh["label"], sc["clean_labels"], K1)
        pos.append(np.asarray(qh["p_occ"], np.float32))
        probes = beam_probes(sc["points"], sc["pose"], step, stride)
        if len(probes):
            neg.append(np.asarray(query(probes)["p_occ"], np.float32))
    per = iou(conf)
    present = conf[1:].sum(1) > 0
    scores = np.concatenate(pos + neg)
    positive = np.zeros(len(scores), bool)
    positive[: sum(len(a) for a in pos)] = True
    return {"iou": per.tolist(), "miou": float(np.nanmean(per[1:][present])) if present.any() else float("nan"),
            "auc": roc_auc(scores, positive), "hits": int(positive.sum()), "free_probes": int((~positive).sum())}
