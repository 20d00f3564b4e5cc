"""Soft labels (reading K15) and per-class length scales (reading K16) on the
GPU against the FP64 oracle.

Soft labels: every hit carries a probability vector over the occupied
classes; groups are (cell, most probable class) and carry the exact mean of
their members' weights per class.  The training set (centroids and weights)
must match the oracle's bit for bit; the map keys and pair counts exactly and
alpha within relative 1e-5.  One-hot vectors reproduce the hard-label update.
Per-class length scales: a class-k point reaches the voxels within
l_k = l * l_scale[k]; keys, pair counts exact, alpha within relative 1e-5.
"""
import numpy as np
import pytest

from synth import scenes

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def sb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_04631_gb300 as sbm
    sbm.load()
    return sbm


def _rel(a, b):
    return np.abs(a.astype(np.float64) - b) / np.abs(b)


def _softmax_probs(labels, K, rng, sharp=3.0):
    """Seeded softmax vectors over classes 1..K peaked at each point's label,
    with exact ties, exact zeros and subnormal entries mixed in."""
    n = len(labels)
    logits = rng.normal(0.0, 1.0, size=(n, K)).astype(np.float32)
    logits[np.arange(n), labels - 1] += np.float32(sharp)
    e = np.exp(logits - logits.max(1, keepdims=True))
    p = (e / e.sum(1, keepdims=True)).astype(np.float32)
    p[::17, :] = 0.0
    p[::17, 0] = 1.0  # one-hot rows
    p[5::23, 1] = p[5::23, 0]  # exact ties: the lower class wins
    p[7::29, -1] = np.float32(1e-42)  # subnormal weights
    p[9::31, 2] = 0.0
    return p


def _params(sb, prm, **kw):
    return sb.default_params(**prm, pool_blocks=1 << 15, sample_capacity=1 << 22, track_pairs=1, device=0, **kw)


def _small_soft_scan(seed=0):
    sc = scenes.small_region_scan(seed)
    K = scenes.SMALL_SCENE_PARAMS["num_classes"]
    probs = _softmax_probs(sc["labels"], K, np.random.default_rng(100 + seed))
    return sc, probs


def _sorted_rows(x, w):
    order = np.lexsort(tuple(w.T[::-1]) + (x[:, 2], x[:, 1], x[:, 0]))
    return x[order], w[order]


def test_soft_training_set_bit_exact(sb, orc):
    sc, probs = _small_soft_scan(0)
    prm = dict(scenes.SMALL_SCENE_PARAMS)
    with sb.Map(_params(sb, prm)) as m:
        gx, gw = m.training_set_soft(sc["points"], probs, sc["pose"])
    ox, ow, ost = orc.soft_training_set(orc.params(**prm), sc["points"], probs, sc["pose"])
    assert len(gx) == len(ox) == ost["train"]
    gx, gw = _sorted_rows(gx, gw)
    ox, ow = _sorted_rows(ox, ow)
    np.testing.assert_array_equal(gx, ox)
    np.testing.assert_array_equal(gw.view(np.uint32), ow.view(np.uint32))


@pytest.mark.parametrize("seed", [0, 1])
def test_soft_map_matches_oracle(sb, orc, seed):
    sc, probs = _small_soft_scan(seed)
    prm = dict(scenes.SMALL_SCENE_PARAMS)
    om = orc.OracleMap(orc.params(**prm))
    ost = om.insert_scan_soft(sc["points"], probs, sc["pose"])
    with sb.Map(_params(sb, prm)) as m:
        st = m.insert_scan_soft(sc["points"], probs, sc["pose"])
        keys, alpha, pairs = m.export(pairs=True)
    okeys, oalpha, opairs = om.export()
    assert st["train_points"] == ost["train"]
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    assert st["pairs"] == int(opairs.sum())
    assert _rel(alpha, oalpha).max() <= RTOL


def test_soft_map_in_the_weighted_form(sb, orc):
    """l = 4.5 voxels: beyond the fast point-major form (offsets -3..3), so soft
    labels take the weighted form (one warp per point over the cube)."""
    sc, probs = _small_soft_scan(2)
    prm = dict(scenes.SMALL_SCENE_PARAMS, length_scale=0.45)
    om = orc.OracleMap(orc.params(**prm))
    om.insert_scan_soft(sc["points"], probs, sc["pose"])
    with sb.Map(_params(sb, prm)) as m:
        m.insert_scan_soft(sc["points"], probs, sc["pose"])
        keys, alpha, pairs = m.export(pairs=True)
    okeys, oalpha, opairs = om.export()
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    assert _rel(alpha, oalpha).max() <= RTOL


def test_one_hot_probabilities_reproduce_the_hard_update(sb):
    sc = scenes.small_region_scan(3)
    prm = dict(scenes.SMALL_SCENE_PARAMS)
    K = prm["num_classes"]
    onehot = np.eye(K, dtype=np.float32)[sc["labels"] - 1]
    with sb.Map(_params(sb, prm)) as ms, sb.Map(_params(sb, prm)) as mh:
        sx, sw = ms.training_set_soft(sc["points"], onehot, sc["pose"])
        hx, hl = mh.training_set(sc["points"], sc["labels"], sc["pose"])
        np.testing.assert_array_equal(sx, hx)
        np.testing.assert_array_equal(sw, np.eye(K + 1, dtype=np.float32)[hl])
        ss = ms.insert_scan_soft(sc["points"], onehot, sc["pose"])
        hs = mh.insert_scan(sc["points"], sc["labels"], sc["pose"])
        assert ss["pairs"] == hs["pairs"] and ss["train_points"] == hs["train_points"]
        for a, b in zip(ms.export(pairs=True), mh.export(pairs=True)):
            if a.dtype == np.float32:
                assert _rel(a, b).max() <= RTOL  # FP32 sums in another order
            else:
                np.testing.assert_array_equal(a, b)


def test_soft_street_scan(sb, orc):
    """A whole 64 x 2048 street scan with softmax vectors over 19 classes."""
    sc = next(scenes.street_sequence(1, first=13))
    prm = dict(scenes.STREET_PARAMS)
    probs = _softmax_probs(sc["labels"], prm["num_classes"], np.random.default_rng(7))
    om = orc.OracleMap(orc.params(**prm))
    om.insert_scan_soft(sc["points"], probs, sc["pose"])
    p = sb.default_params(**prm, pool_blocks=1 << 16, sample_capacity=1 << 23, track_pairs=1, device=0)
    with sb.Map(p) as m:
        m.insert_scan_soft(sc["points"], probs, sc["pose"])
        keys, alpha, pairs = m.export(pairs=True)
    okeys, oalpha, opairs = om.export()
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    assert _rel(alpha, oalpha).max() <= RTOL


def test_soft_labels_refusals_leave_the_map_unchanged(sb):
    sc, probs = _small_soft_scan(4)
    prm = dict(scenes.SMALL_SCENE_PARAMS)
    with sb.Map(_params(sb, prm)) as m:
        m.insert_scan_soft(sc["points"], probs, sc["pose"])
        before = m.export(pairs=True)
        for bad in (np.where(np.arange(probs.size).reshape(probs.shape) == 3, -0.1, probs),
                    np.where(np.arange(probs.size).reshape(probs.shape) == 5, 1.5, probs),
                    np.where(np.arange(len(probs))[:, None] == 8, 0.0, probs),
                    np.where(np.arange(probs.size).reshape(probs.shape) == 11, np.nan, probs)):
            with pytest.raises(sb.SbkiError) as e:
                m.insert_scan_soft(sc["points"], bad.astype(np.float32), sc["pose"])
            assert e.value.status == sb.ERR_LABEL_RANGE
        after = m.export(pairs=True)
        for a, b in zip(before, after):
            np.testing.assert_array_equal(a, b)
    for kw in (dict(accumulate_mode=1), dict(association=1)):
        with sb.Map(_params(sb, prm, **kw)) as m:
            with pytest.raises(sb.SbkiError) as e:
                m.insert_scan_soft(sc["points"], probs, sc["pose"])
            assert e.value.status == sb.ERR_INVALID_ARG


# ------------------------------------------------------------ per-class length scales

# supports in voxels: (2.5, 1.5, 3.5, 2.25) and (3, 2.5, 1.25, 3.625): the fast point-major form takes the
# classes whose support needs at most 7 offsets per axis, the weighted form the others; (2.5, 0.75, 3, 2.5):
# a support below half the voxel diagonal sends every class to the weighted form
@pytest.mark.parametrize("seed,ls", [(0, [1.0, 0.6, 1.4, 0.9]), (1, [1.2, 1.0, 0.5, 1.45]), (2, [1.0, 0.3, 1.2, 1.0])])
def test_per_class_length_scale_matches_oracle(sb, orc, seed, ls):
    rng = np.random.default_rng(seed)
    n = 1200
    xyz = rng.uniform(-1.3, 1.3, size=(n, 3)).astype(np.float32)
    xyz[: n // 10] = (np.round(xyz[: n // 10] / 0.1) * 0.1).astype(np.float32)
    lab = rng.integers(0, 4, size=n).astype(np.int32)
    prm = dict(res=0.1, length_scale=0.25, sigma0=0.6, alpha0=0.001, num_classes=3)
    p = _params(sb, prm)
    sb.set_param(p, "l_scale", ls)
    om = orc.OracleMap(orc.params(**prm, l_scale=ls))
    om.insert_training(xyz, lab)
    with sb.Map(p) as m:
        st = m.insert_training(xyz, lab)
        keys, alpha, pairs = m.export(pairs=True)
    okeys, oalpha, opairs = om.export()
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    assert st["pairs"] == int(opairs.sum())
    assert _rel(alpha, oalpha).max() <= RTOL


def test_per_class_length_scale_scan_and_refusals(sb, orc):
    sc = scenes.small_region_scan(5)
    prm = dict(scenes.SMALL_SCENE_PARAMS)
    K = prm["num_classes"]
    ls = [1.0 + 0.1 * ((k % 5) - 2) for k in range(K + 1)]
    p = _params(sb, prm)
    sb.set_param(p, "l_scale", ls)
    om = orc.OracleMap(orc.params(**prm, l_scale=ls))
    om.insert_scan(sc["points"], sc["labels"], sc["pose"])
    with sb.Map(p) as m:
        m.insert_scan(sc["points"], sc["labels"], sc["pose"])
        keys, alpha, pairs = m.export(pairs=True)
        xyz, lab = m.training_set(sc["points"], sc["labels"], sc["pose"])
        m.grad_clear()
        with pytest.raises(sb.SbkiError) as e:
            m.backward(np.concatenate([xyz, lab[:, None].astype(np.float32)], 1))
        assert e.value.status == sb.ERR_INVALID_ARG
    okeys, oalpha, opairs = om.export()
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    assert _rel(alpha, oalpha).max() <= RTOL
    for kw in (dict(accumulate_mode=1), dict(association=1)):
        q = _params(sb, prm, **kw)
        sb.set_param(q, "l_scale", ls)
        with pytest.raises(sb.SbkiError) as e:
            sb.Map(q)
        assert e.value.status == sb.ERR_INVALID_ARG
