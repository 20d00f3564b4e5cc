"""Batched form: several scans, each into its own map of one handle (or two
into the same map), in one pass of the device pipeline recorded as a CUDA
graph.  Every map must equal the FP64 oracle map fed the same scans (keys and
pair counts exact, alpha within relative 1e-5), also on a replay of the
recorded graph, and equal the maps built by one sbki_insert_scan per scan.
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


PRM = dict(scenes.BATCH_PARAMS, num_classes=19)


def _params(sb, num_maps, **kw):
    p = sb.default_params(res=PRM["res"], length_scale=PRM["length_scale"], sigma0=PRM["sigma0"], alpha0=PRM["alpha0"],
                          free_step=PRM["free_step"], num_classes=PRM["num_classes"], min_range=PRM["min_range"],
                          max_range=PRM["max_range"], pool_blocks=1 << 15, sample_capacity=1 << 22, track_pairs=1,
                          num_maps=num_maps, device=0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.fixture(scope="module")
def scans():
    return scenes.batch_scans(n_maps=5, n_min=1500, n_max=4000)


def _as_batch(scans, maps, device_every=2):
    import torch
    out = []
    for i, (sc, mid) in enumerate(zip(scans, maps)):
        pts, lab = sc["points"], sc["labels"]
        if i % device_every == 0:  # mix device and host inputs
            pts, lab = torch.from_numpy(pts).cuda(), torch.from_numpy(lab).cuda()
        out.append(dict(points=pts, labels=lab, pose=sc["pose"], map_id=mid))
    return out


def _assert_map_equal(m, map_id, om):
    m.select(map_id)
    keys, alpha, pairs = m.export(pairs=True)
    okeys, oalpha, opairs = om.export()
    assert keys.shape == okeys.shape, (map_id, keys.shape, okeys.shape)
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    rel = np.abs(alpha.astype(np.float64) - oalpha) / np.abs(oalpha)
    assert rel.max(initial=0.0) <= RTOL, (map_id, rel.max())


def test_batch_into_separate_maps_matches_oracle_and_replays(sb, orc, scans):
    import torch
    m = sb.Map(_params(sb, 6))
    st = m.insert_batch(_as_batch(scans, range(5)))
    oms = [orc.OracleMap(orc.params(**PRM)) for _ in range(5)]
    ost = [om.insert_scan(sc["points"], sc["labels"], sc["pose"]) for om, sc in zip(oms, scans)]
    assert st["hits"] == sum(o["hits"] for o in ost)
    assert st["train_points"] == sum(o["train"] for o in ost)
    for i, om in enumerate(oms):
        _assert_map_equal(m, i, om)
    m.select(5)
    assert m.voxel_count() == 0
    # a second batch of the same size replays the recording; scans go to other maps now
    shifted = [scans[(i + 1) % 5] for i in range(5)]
    m.insert_batch(_as_batch(shifted, range(5), device_every=3))
    for i, om in enumerate(oms):
        om.insert_scan(shifted[i]["points"], shifted[i]["labels"], shifted[i]["pose"])
        _assert_map_equal(m, i, om)
    torch.cuda.synchronize()


def test_two_scans_into_one_map_and_sequential_equivalence(sb, orc, scans):
    m = sb.Map(_params(sb, 2))
    m.insert_batch(_as_batch(scans[:3], [0, 1, 0]))
    om0 = orc.OracleMap(orc.params(**PRM))
    om0.insert_scan(scans[0]["points"], scans[0]["labels"], scans[0]["pose"])
    om0.insert_scan(scans[2]["points"], scans[2]["labels"], scans[2]["pose"])
    om1 = orc.OracleMap(orc.params(**PRM))
    om1.insert_scan(scans[1]["points"], scans[1]["labels"], scans[1]["pose"])
    _assert_map_equal(m, 0, om0)
    _assert_map_equal(m, 1, om1)
    # the same scans one call each, into the selected map of a second handle
    seq = sb.Map(_params(sb, 2))
    for sc, mid in zip(scans[:3], [0, 1, 0]):
        seq.select(mid)
        seq.insert_scan(sc["points"], sc["labels"], sc["pose"])
    for mid in (0, 1):
        m.select(mid)
        seq.select(mid)
        k1, a1, p1 = m.export(pairs=True)
        k2, a2, p2 = seq.export(pairs=True)
        np.testing.assert_array_equal(k1, k2)
        np.testing.assert_array_equal(p1, p2)
        np.testing.assert_allclose(a1, a2, rtol=RTOL)
    # queries read the selected map: at voxel centres, probs = alpha / sum(alpha)
    m.select(1)
    k1, a1, _ = m.export()
    step = max(1, len(k1) // 50)
    centres = ((k1[::step] + 0.5) * PRM["res"]).astype(np.float32)
    q = m.query(centres, var=False, mode=False)
    a = a1[::step].astype(np.float64)
    np.testing.assert_allclose(q["probs"], a / a.sum(1, keepdims=True), rtol=1e-5)


def test_batch_errors_leave_maps_unchanged(sb, scans):
    m = sb.Map(_params(sb, 2))
    m.insert_batch(_as_batch(scans[:2], [0, 1]))
    m.select(0)
    k0, a0, _ = m.export()
    with pytest.raises(sb.SbkiError) as e:
        m.insert_batch(_as_batch(scans[:2], [0, 2]))
    assert e.value.status == sb.ERR_INVALID_ARG
    # too many samples for the per-update capacity: nothing changes
    small = sb.Map(_params(sb, 2, sample_capacity=1 << 14))
    with pytest.raises(sb.SbkiError) as e:
        small.insert_batch(_as_batch(scans[:2], [0, 1]))
    assert e.value.status == sb.ERR_CAPACITY
    small.select(0)
    assert small.voxel_count() == 0
    m.select(0)
    k1, a1, _ = m.export()
    np.testing.assert_array_equal(k0, k1)
    np.testing.assert_array_equal(a0, a1)


def test_tuning_changes_speed_not_results(sb, scans):
    from paper_1909_04631_gb300 import autotune
    outs = []
    for tune in (dict(accumulate_ctas_per_sm=1, accumulate_chunk=1, touch_ctas_per_sm=1, ingest_ctas_per_sm=1),
                 dict(accumulate_ctas_per_sm=0, accumulate_chunk=16, touch_ctas_per_sm=8, ingest_ctas_per_sm=16)):
        m = sb.Map(_params(sb, 3))
        m.set_tuning(**tune)
        assert m.get_tuning() == tune
        m.insert_batch(_as_batch(scans[:3], [0, 1, 2]))
        m.insert_batch(_as_batch(scans[2:5], [0, 1, 2]))  # replays the recording made with this tuning
        outs.append([(m.select(i), m.export(pairs=True))[1] for i in range(3)])
    for (k1, a1, p1), (k2, a2, p2) in zip(*outs):
        np.testing.assert_array_equal(k1, k2)
        np.testing.assert_array_equal(p1, p2)
        np.testing.assert_allclose(a1, a2, rtol=RTOL)
    res = autotune.autotune(_params(sb, 3), _as_batch(scans[:3], [0, 1, 2]),
                            candidates=dict(accumulate_ctas_per_sm=(0, 2), accumulate_chunk=(4,), touch_ctas_per_sm=(8,),
                                            ingest_ctas_per_sm=(16,)), reps=1)
    # two shapes in each accumulation form, and the library's default shape timed beside them
    assert len(res["trials"]) == 4 and res["tuning"] in [t for t, _ in res["trials"]] and res["ms"] > 0
    assert {t["accumulate_mode"] for t, _ in res["trials"]} == {0, 1} and res["default_ms"] > 0
    shapes, mode = autotune.split_tuning(res["tuning"])
    assert mode in (0, 1) and "accumulate_mode" not in shapes
    with pytest.raises(sb.SbkiError):
        sb.Map(_params(sb, 1)).set_tuning(accumulate_chunk=0)


@pytest.mark.parametrize("rule", ["l_scale", "association", "sigma0_scale"])
def test_batch_under_the_other_map_rules(sb, orc, scans, rule):
    """The recorded update with per-class length scales (fast and weighted
    forms in one graph), the extended-block association, or per-class kernel
    scales: every map against the oracle, also after a replay."""
    K1 = PRM["num_classes"] + 1
    vals = [1.0 + 0.25 * ((k % 5) - 2) / 2.0 for k in range(K1)]  # 0.75 .. 1.25: some supports above 7 offsets
    p = _params(sb, 3)
    oprm = dict(PRM)
    if rule == "association":
        p.association = 1
        oprm["association"] = 1
    else:
        sb.set_param(p, rule, vals)
        oprm[rule] = vals
    batch = _as_batch(scans[:3], [0, 1, 2])
    oms = []
    for sc in scans[:3]:
        om = orc.OracleMap(orc.params(**oprm))
        om.insert_scan(sc["points"], sc["labels"], sc["pose"])
        oms.append(om)
    with sb.Map(p) as m:
        m.insert_batch(batch)
        for i, om in enumerate(oms):
            _assert_map_equal(m, i, om)
        m.insert_batch(batch)  # replay: the same increments again
        for i, om in enumerate(oms):
            m.select(i)
            keys, alpha, pairs = m.export(pairs=True)
            okeys, oalpha, opairs = om.export()
            np.testing.assert_array_equal(keys, okeys)
            np.testing.assert_array_equal(pairs, 2 * opairs)
            a0 = PRM["alpha0"]
            rel = np.abs((alpha.astype(np.float64) - a0) - 2 * (oalpha - a0)) / (oalpha - a0 + 1e-30)
            assert rel[oalpha > 2 * a0].max(initial=0.0) <= 2e-5
