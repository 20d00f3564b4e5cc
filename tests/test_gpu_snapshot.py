"""Snapshot and resume: sbki_export, then sbki_import into another map (or another
map of a multi-map handle), gives the same keys, alpha within one FP32 rounding,
the same read-off, and further updates continue as on the original map."""
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


def _params(sb, **kw):
    prm = dict(scenes.SMALL_SCENE_PARAMS)
    p = sb.default_params(res=prm["res"], length_scale=prm["length_scale"], sigma0=prm["sigma0"], alpha0=prm["alpha0"],
                          free_step=prm["free_step"], num_classes=prm["num_classes"], max_range=prm["max_range"],
                          pool_blocks=1 << 14, sample_capacity=1 << 22, device=0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_export_import_roundtrip_and_resume(sb):
    scans = [scenes.small_region_scan(s, n_az=60, n_el=40) for s in range(2)]
    a = sb.Map(_params(sb))
    a.insert_scan(scans[0]["points"], scans[0]["labels"], scans[0]["pose"])
    keys, alpha, _ = a.export()
    b = sb.Map(_params(sb, num_maps=3))
    b.select(2)
    b.import_(keys, alpha)
    k2, a2, _ = b.export()
    np.testing.assert_array_equal(k2, keys)
    np.testing.assert_allclose(a2, alpha, rtol=5e-7)  # two FP32 roundings
    b.select(0)
    assert b.voxel_count() == 0
    # read-off of the restored map
    b.select(2)
    centres = ((keys[::97] + 0.5) * scenes.SMALL_SCENE_PARAMS["res"]).astype(np.float32)
    qa, qb = a.query(centres), b.query(centres)
    np.testing.assert_allclose(qb["probs"], qa["probs"], rtol=1e-6, atol=1e-9)
    # a voxel whose exported alpha is exactly the prior lost its (sub-ulp) mass
    # in the export: restored, it has no kernel mass and reads as unknown
    informative = ~np.all(alpha[::97] == np.float32(scenes.SMALL_SCENE_PARAMS["alpha0"]), axis=1)
    np.testing.assert_array_equal(qb["state"][informative], qa["state"][informative])
    assert np.all(qb["state"][~informative] == 1)
    # resume: the next scan on both
    a.insert_scan(scans[1]["points"], scans[1]["labels"], scans[1]["pose"])
    b.insert_scan(scans[1]["points"], scans[1]["labels"], scans[1]["pose"])
    k3, a3, _ = a.export()
    k4, a4, _ = b.export()
    np.testing.assert_array_equal(k3, k4)
    np.testing.assert_allclose(a4, a3, rtol=1e-5)
    # importing over existing voxels overwrites them
    b.import_(keys[:10], np.full((10, alpha.shape[1]), 0.5, np.float32))
    qk = ((keys[:10] + 0.5) * scenes.SMALL_SCENE_PARAMS["res"]).astype(np.float32)
    np.testing.assert_allclose(b.query(qk)["probs"], 1.0 / alpha.shape[1], rtol=1e-6)


def test_device_export_in_pool_order_equals_the_sorted_export(sb):
    """sbki_export_blocks (device rows in pool order) holds exactly the rows of
    sbki_export (host, sorted by key), for the selected map of a multi-map
    handle, into device and into host buffers."""
    import torch
    scans = [scenes.small_region_scan(s, n_az=50, n_el=30) for s in range(2)]
    m = sb.Map(_params(sb, num_maps=2))
    for i, sc in enumerate(scans):
        m.select(i)
        m.insert_scan(sc["points"], sc["labels"], sc["pose"])
    for i in range(2):
        m.select(i)
        keys, alpha, _ = m.export()
        dk, da = m.export_blocks(device=torch.device("cuda", 0))
        hk, ha = m.export_blocks()
        assert dk.is_cuda and da.is_cuda
        np.testing.assert_array_equal(dk.cpu().numpy(), hk)
        np.testing.assert_array_equal(da.cpu().numpy(), ha)
        order = np.lexsort((hk[:, 2], hk[:, 1], hk[:, 0]))
        np.testing.assert_array_equal(hk[order], keys)
        np.testing.assert_array_equal(ha[order], alpha)
    m.close()
