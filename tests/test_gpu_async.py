"""Scans streamed through sbki_insert_scan_async (the form bench.py times):
the same map as synchronous inserts (keys and pair counts exact, alpha up to
the order of FP32 sums), stage times of every asynchronous insert counted at
the next synchronising call (two sets of events), a profile reset dropping an
insert not yet read, and a device-side error surfacing with the map unchanged."""
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


@pytest.fixture(scope="module")
def scans():
    return [scenes.small_region_scan(s) for s in range(4)]


def _params(sb):
    return sb.default_params(**scenes.SMALL_SCENE_PARAMS, pool_blocks=1 << 14, sample_capacity=1 << 21,
                             track_pairs=1, device=0)


def _rel(a, b):
    return np.abs(a.astype(np.float64) - b) / np.maximum(np.abs(b.astype(np.float64)), 1e-30)


def test_async_inserts_equal_synchronous_ones(sb, scans):
    import torch
    dp = [torch.from_numpy(s["points"]).cuda() for s in scans]
    dl = [torch.from_numpy(s["labels"]).cuda() for s in scans]
    with sb.Map(_params(sb)) as ma, sb.Map(_params(sb)) as ms:
        last = None
        for s, p, l in zip(scans, dp, dl):
            assert ma.insert_scan(p, l, s["pose"], sync=False) is None
            last = ms.insert_scan(p, l, s["pose"])
        st = ma.sync()
        assert st["pairs"] == last["pairs"] and st["train_points"] == last["train_points"]
        ka, aa, pa = ma.export(pairs=True)
        ks, as_, ps = ms.export(pairs=True)
    np.testing.assert_array_equal(ka, ks)
    np.testing.assert_array_equal(pa, ps)
    assert _rel(aa, as_).max() <= 1e-5


def test_async_stage_times_are_all_counted(sb, scans):
    import torch
    dp = [torch.from_numpy(s["points"]).cuda() for s in scans]
    dl = [torch.from_numpy(s["labels"]).cuda() for s in scans]
    with sb.Map(_params(sb)) as m:
        m.insert_scan(dp[0], dl[0], scans[0]["pose"])
        m.profile(True, reset=True)
        for s, p, l in zip(scans, dp, dl):
            m.insert_scan(p, l, s["pose"], sync=False)
        m.sync()
        pr = m.profile_read()
        assert pr["inserts"] == len(scans)
        assert pr["ingest_ms"] > 0 and pr["blocks_ms"] > 0 and pr["accumulate_ms"] > 0
        assert pr["readback_bytes"] > 0
        # mixed: synchronous after asynchronous
        m.profile(True, reset=True)
        m.insert_scan(dp[1], dl[1], scans[1]["pose"], sync=False)
        m.insert_scan(dp[2], dl[2], scans[2]["pose"])
        assert m.profile_read()["inserts"] == 2
        # a reset drops an asynchronous insert not yet read
        m.insert_scan(dp[3], dl[3], scans[3]["pose"], sync=False)
        m.profile(True, reset=True)
        m.sync()
        assert m.profile_read()["inserts"] == 0
        m.profile(False, reset=True)


def test_async_error_surfaces_and_leaves_the_map_unchanged(sb, scans):
    with sb.Map(_params(sb)) as m:
        m.insert_scan(scans[0]["points"], scans[0]["labels"], scans[0]["pose"])
        before = m.export(pairs=True)
        bad = scans[1]["labels"].copy()
        bad[7] = 99
        with pytest.raises(sb.SbkiError) as e:
            m.insert_scan(scans[1]["points"], bad, scans[1]["pose"], sync=False)
            m.sync()
        assert e.value.status == sb.ERR_LABEL_RANGE
        after = m.export(pairs=True)
        for a, b in zip(before, after):
            np.testing.assert_array_equal(a, b)
