"""Parity of the counting sensor model (S-CSM, Eq. alpha) on the GPU with the
FP64 oracle, through the C ABI.

Counts are integers, so the voxel keys, every class's count in every voxel and
the pair counts must match exactly; alpha (prior included) to the FP32
rounding of alpha0 + count; read-off labels exactly (equal counts tie in both).
"""
import numpy as np
import pytest

from synth import scenes

pytestmark = pytest.mark.gpu

RTOL = 1e-6  # alpha0 + count rounded to FP32


@pytest.fixture(scope="module")
def sb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_04631_gb300 as sbm
    sbm.load()
    return sbm


def _params(sb, prm, **kw):
    p = sb.default_params(res=prm["res"], length_scale=prm.get("length_scale", 0.3), sigma0=prm.get("sigma0", 0.1),
                          alpha0=prm["alpha0"], free_step=prm.get("free_step", 0.3), num_classes=prm["num_classes"],
                          min_range=prm.get("min_range", 0.0), max_range=prm.get("max_range", 100.0),
                          block_edge=prm.get("block_edge", 8), pool_blocks=1 << 15, sample_capacity=1 << 22,
                          track_pairs=1, device=0, sensor_model=1)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _orc_params(orc, prm):
    return orc.params(**dict(prm, sensor_model=1))


def _assert_counts_equal(m, om, a0):
    keys, alpha, pairs = m.export(pairs=True)
    okeys, oalpha, opairs = om.export()
    assert keys.shape == okeys.shape
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    np.testing.assert_array_equal(np.rint(alpha.astype(np.float64) - np.float32(a0)), np.rint(oalpha - a0))
    rel = np.abs(alpha.astype(np.float64) - oalpha) / oalpha
    assert rel.max(initial=0.0) <= RTOL
    return keys, oalpha, opairs


@pytest.mark.parametrize("seed,n,res,K,edge,shift", [(0, 300, 0.1, 3, 8, 0.0), (1, 4000, 0.1, 19, 8, 0.0),
                                                     (2, 900, 0.05, 11, 4, 0.0), (3, 1, 0.1, 2, 8, 0.0),
                                                     (4, 2000, 0.1, 5, 8, 20411.05)])
def test_counting_training_sets_match_oracle(sb, orc, seed, n, res, K, edge, shift):
    """Random clouds (a tenth of them on voxel faces, negative and far-off
    coordinates): the voxel each point counts in is the read-off's key."""
    rng = np.random.default_rng(seed)
    xyz = (rng.uniform(-1.7, 1.9, size=(n, 3)) + shift).astype(np.float32)
    xyz[: n // 10] = (np.round(xyz[: n // 10] / res) * res).astype(np.float32)
    lab = rng.integers(0, K + 1, size=n).astype(np.int32)
    prm = dict(res=res, length_scale=3 * res, alpha0=0.001, num_classes=K, block_edge=edge)
    m = sb.Map(_params(sb, prm))
    st = m.insert_training(xyz, lab)
    om = orc.OracleMap(_orc_params(orc, prm))
    om.insert_training(xyz, lab)
    _, _, pairs = _assert_counts_equal(m, om, 0.001)
    assert st["pairs"] == n == int(pairs.sum())
    assert st["total_blocks"] == len(om.block_keys())


def test_counting_scans_match_oracle_and_stats(sb, orc):
    prm = dict(scenes.SMALL_SCENE_PARAMS)
    m = sb.Map(_params(sb, prm))
    om = orc.OracleMap(_orc_params(orc, prm))
    for k in range(3):
        sc = scenes.small_region_scan(k)
        st = m.insert_scan(sc["points"], sc["labels"], sc["pose"])
        ost = om.insert_scan(sc["points"], sc["labels"], sc["pose"])
        assert (st["hits"], st["free_samples"], st["train_points"]) == (ost["hits"], ost["free"], ost["train"])
        assert st["pairs"] == ost["train"]
        if k == 0:
            assert st["touched_blocks"] == st["new_blocks"] == len(om.block_keys())
    keys, oalpha, _ = _assert_counts_equal(m, om, prm["alpha0"])
    # read-off at every voxel centre of the map and at the last scan's hits (world frame)
    T = sc["pose"]
    hits = (sc["points"][:2000].astype(np.float64) @ T[:3, :3].T + T[:3, 3]).astype(np.float32)
    q = np.concatenate([((keys + 0.5) * prm["res"]).astype(np.float32), hits])
    g = m.query(q)
    o = om.query(q)
    np.testing.assert_allclose(g["probs"], o["probs"], rtol=1e-5, atol=1e-7)
    np.testing.assert_array_equal(g["label"], o["label"])
    near = (np.abs(o["p_occ"] - prm.get("free_thresh", 0.47)) < 1e-5) | (np.abs(o["p_occ"] - 0.6) < 1e-5)
    np.testing.assert_array_equal(g["state"][~near], o["state"][~near])


def test_counting_batch_matches_oracle(sb, orc):
    import torch
    prm = dict(scenes.BATCH_PARAMS, num_classes=19)
    scans = scenes.batch_scans(n_maps=4, n_min=1500, n_max=4000)
    m = sb.Map(_params(sb, prm, num_maps=3))
    maps = [0, 1, 2, 0]
    batch = []
    for i, (sc, mid) in enumerate(zip(scans, maps)):
        pts, lab = sc["points"], sc["labels"]
        if i % 2 == 0:
            pts, lab = torch.from_numpy(pts).cuda(), torch.from_numpy(lab).cuda()
        batch.append(dict(points=pts, labels=lab, pose=sc["pose"], map_id=mid))
    st = m.insert_batch(batch)
    oms = [orc.OracleMap(_orc_params(orc, prm)) for _ in range(3)]
    ost = [oms[mid].insert_scan(sc["points"], sc["labels"], sc["pose"]) for sc, mid in zip(scans, maps)]
    assert st["train_points"] == st["pairs"] == sum(o["train"] for o in ost)
    for i, om in enumerate(oms):
        m.select(i)
        _assert_counts_equal(m, om, prm["alpha0"])
    torch.cuda.synchronize()


def test_counting_capacity_leaves_map_unchanged(sb):
    prm = dict(res=0.1, alpha0=0.001, num_classes=3)
    rng = np.random.default_rng(5)
    xyz = rng.uniform(-0.5, 0.5, size=(200, 3)).astype(np.float32)
    lab = rng.integers(0, 4, size=200).astype(np.int32)
    m = sb.Map(_params(sb, prm, pool_blocks=8))
    m.insert_training(xyz, lab)
    before = m.export(pairs=True)
    far = (xyz * 40.0).astype(np.float32)  # needs far more than 8 blocks
    with pytest.raises(sb.SbkiError) as e:
        m.insert_training(far, lab)
    assert e.value.status == sb.ERR_CAPACITY
    after = m.export(pairs=True)
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)


def test_counting_model_refuses_backward_and_block_major(sb):
    prm = dict(res=0.1, alpha0=0.001, num_classes=3)
    m = sb.Map(_params(sb, prm))
    xyzl = np.array([[0.05, 0.05, 0.05, 1.0]], np.float32)
    m.insert_training(xyzl[:, :3], xyzl[:, 3].astype(np.int32))
    m.grad_clear()
    with pytest.raises(sb.SbkiError) as e:
        m.backward(xyzl)
    assert e.value.status == sb.ERR_INVALID_ARG
    with pytest.raises(sb.SbkiError) as e:
        sb.Map(_params(sb, prm, accumulate_mode=1))
    assert e.value.status == sb.ERR_INVALID_ARG


def test_counting_full_street_scan_matches_oracle(sb, orc):
    """One full 64 x 2048 LiDAR street scan (about 130k hits, 2.9M free samples)
    in the benchmark's map configuration: the whole counting map, every voxel
    of every block, equals the oracle's."""
    sc = next(scenes.street_sequence(1, first=5))
    prm = dict(scenes.STREET_PARAMS)
    m = sb.Map(_params(sb, prm, pool_blocks=1 << 18, sample_capacity=1 << 23))
    st = m.insert_scan(sc["points"], sc["labels"], sc["pose"])
    om = orc.OracleMap(_orc_params(orc, prm))
    ost = om.insert_scan(sc["points"], sc["labels"], sc["pose"])
    assert (st["hits"], st["free_samples"], st["train_points"]) == (ost["hits"], ost["free"], ost["train"])
    assert st["pairs"] == ost["train"] and st["touched_blocks"] == len(om.block_keys())
    _assert_counts_equal(m, om, prm["alpha0"])
