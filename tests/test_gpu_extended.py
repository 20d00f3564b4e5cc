"""Extended-block association (Sec. IV, the paper's software; reading K14) on
the GPU against the FP64 oracle with association 1: a voxel of block b takes
only the training points whose own voxel lies in b or one of its six face
neighbours.  Keys and pair counts exact, alpha within relative 1e-5, in both
accumulation forms, on clouds placed around block edges and corners and on a
whole 64 x 2048 street scan; the differentiable entry points refuse it.
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


def _compare(m, om):
    keys, alpha, pairs = m.export(pairs=True)
    okeys, oalpha, opairs = om.export()
    assert keys.shape == okeys.shape
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    assert _rel(alpha, oalpha).max(initial=0.0) <= RTOL
    return keys, pairs


@pytest.mark.parametrize("mode", [0, 1], ids=["point_major", "block_major"])
@pytest.mark.parametrize("B,l,seed", [(8, 0.3, 31), (4, 0.3, 32), (8, 0.25, 33), (8, 0.5, 34)])
def test_extended_block_clouds(sb, orc, mode, B, l, seed):
    rng = np.random.default_rng(seed)
    res, n = 0.1, 900
    xyz = (np.round(rng.uniform(-1.2, 1.2, size=(n, 3)) / (B * res)) * (B * res)
           + rng.uniform(-0.12, 0.12, size=(n, 3))).astype(np.float32)  # around block corners and edges
    lab = rng.integers(0, 5, size=n).astype(np.int32)
    prm = dict(res=res, length_scale=l, sigma0=0.37, alpha0=0.001, num_classes=4, block_edge=B)
    p = sb.default_params(**prm, pool_blocks=1 << 14, sample_capacity=1 << 20, track_pairs=1, accumulate_mode=mode,
                          association=1, device=0)
    om = orc.OracleMap(orc.params(**prm, association=1))
    om.insert_training(xyz, lab)
    with sb.Map(p) as m:
        st = m.insert_training(xyz, lab)
        keys, pairs = _compare(m, om)
    assert st["pairs"] == int(pairs.sum())
    # the exact association has strictly more pairs on these clouds
    ex = orc.OracleMap(orc.params(**prm))
    ex.insert_training(xyz, lab)
    assert ex.export()[2].sum() > pairs.sum()


def test_extended_block_street_scan(sb, orc):
    sc = next(scenes.street_sequence(1, first=11))
    prm = dict(scenes.STREET_PARAMS)
    p = sb.default_params(**prm, pool_blocks=1 << 16, sample_capacity=1 << 23, track_pairs=1, association=1,
                          device=0)
    om = orc.OracleMap(orc.params(**prm, association=1))
    om.insert_scan(sc["points"], sc["labels"], sc["pose"])
    with sb.Map(p) as m:
        st = m.insert_scan(sc["points"], sc["labels"], sc["pose"])
        keys, pairs = _compare(m, om)
    assert len(keys) > 2_000_000 and st["pairs"] == int(pairs.sum())


def test_extended_block_refused_by_the_backward_pass(sb):
    prm = dict(scenes.DIFF_PARAMS)
    p = sb.default_params(**prm, pool_blocks=1 << 12, sample_capacity=1 << 18, association=1, device=0)
    rng = np.random.default_rng(5)
    xyz = rng.uniform(-0.5, 0.5, size=(200, 3)).astype(np.float32)
    lab = rng.integers(0, 3, size=200).astype(np.int32)
    xyzl = np.concatenate([xyz, lab[:, None].astype(np.float32)], 1)
    with sb.Map(p) as m:
        m.insert_training(xyz, lab)
        m.grad_clear()
        with pytest.raises(sb.SbkiError) as e:
            m.backward(xyzl)
        assert e.value.status == sb.ERR_INVALID_ARG
    bad = sb.default_params(**prm, association=2, device=0)
    with pytest.raises(sb.SbkiError) as e:
        sb.Map(bad)
    assert e.value.status == sb.ERR_INVALID_ARG
