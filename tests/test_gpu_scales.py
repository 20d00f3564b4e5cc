"""Per-class kernel scales (class k's kernel is sigma0 * sigma0_scale[k] * f)
in every accumulation form against the FP64 oracle: voxel keys and pair counts
exact, alpha within relative 1e-5.  Covers the fast point-major form
(2R + 1 <= 7), the general point-major form (a longer l), the block-major
form and a whole scan; all scales 1 gives the unscaled map (up to the order
of the FP32 reductions)."""
import numpy as np
import pytest

from synth import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_04631_gb300 as sbm
    sbm.load()
    return sbm


def _map(sb, prm, scale, **kw):
    p = sb.default_params(res=prm["res"], length_scale=prm["length_scale"], sigma0=prm["sigma0"], alpha0=prm["alpha0"],
                          free_step=prm.get("free_step", 0.3), num_classes=prm["num_classes"],
                          max_range=prm.get("max_range", 100.0), pool_blocks=1 << 15, sample_capacity=1 << 22,
                          track_pairs=1, device=0, sigma0_scale=scale, **kw)
    return sb.Map(p)


def _assert_equal(m, om):
    keys, alpha, pairs = m.export(pairs=True)
    okeys, oalpha, opairs = om.export()
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    rel = np.abs(alpha.astype(np.float64) - oalpha) / oalpha
    assert rel.max(initial=0.0) <= 1e-5


@pytest.mark.parametrize("l,mode", [(0.3, 0), (0.45, 0), (0.3, 1)], ids=["fast", "general", "block_major"])
def test_class_scales_match_oracle(sb, orc, l, mode):
    rng = np.random.default_rng(37)
    xyz = rng.uniform(-1.2, 1.3, size=(1500, 3)).astype(np.float32)
    lab = rng.integers(0, 6, size=1500).astype(np.int32)
    scale = [0.25, 1.0, 3.0, 0.5, 7.5, 1.75]
    prm = dict(res=0.1, length_scale=l, sigma0=0.4, alpha0=0.001, num_classes=5)
    m = _map(sb, prm, scale, accumulate_mode=mode)
    m.insert_training(xyz, lab)
    om = orc.OracleMap(orc.params(**dict(prm, sigma0_scale=scale)))
    om.insert_training(xyz, lab)
    _assert_equal(m, om)


def test_class_scales_on_a_scan_and_unit_scales(sb, orc):
    sc = scenes.small_region_scan(0, n_az=60, n_el=40)
    prm = dict(scenes.SMALL_SCENE_PARAMS)
    scale = [1.0 + 0.1 * k for k in range(prm["num_classes"] + 1)]
    m = _map(sb, prm, scale)
    m.insert_scan(sc["points"], sc["labels"], sc["pose"])
    om = orc.OracleMap(orc.params(**dict(prm, sigma0_scale=scale)))
    om.insert_scan(sc["points"], sc["labels"], sc["pose"])
    _assert_equal(m, om)
    ones = _map(sb, prm, [1.0] * (prm["num_classes"] + 1))
    plain = _map(sb, prm, [])
    for mm in (ones, plain):
        mm.insert_scan(sc["points"], sc["labels"], sc["pose"])
    (k1, al1, p1), (k2, al2, p2) = ones.export(pairs=True), plain.export(pairs=True)
    np.testing.assert_array_equal(k1, k2)
    np.testing.assert_array_equal(p1, p2)
    # the same map up to the order of the FP32 reductions (not deterministic)
    np.testing.assert_allclose(al1, al2, rtol=2e-6)


def test_class_scales_must_be_positive(sb):
    prm = dict(res=0.1, length_scale=0.3, sigma0=0.4, alpha0=0.001, num_classes=3)
    for bad in ([1.0, 0.0], [1.0, 1.0, float("nan")], [1.0, 1.0, 1.0, -2.0]):
        with pytest.raises(sb.SbkiError) as e:
            _map(sb, prm, bad)
        assert e.value.status == sb.ERR_INVALID_ARG
