"""Map quality (IoU of labels at the scans' hits, occupancy AUC) of maps built
on the GPU against the same scores of the FP64 oracle's maps, for both sensor
models, on a reduced LiDAR street sequence.  The counting model's read-off is
exact (integer counts), so its scores must agree to rounding; the kernel
model's alpha agrees to 1e-5 relative, which can swap near-tied scores.
The read-off adds the prior in FP32 on the GPU and in FP64 in the oracle, so
even counting-model scores may differ by an FP32 rounding."""
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


@pytest.mark.parametrize("model", [1, 0], ids=["counting", "kernel"])
def test_map_quality_matches_oracle(sb, orc, model):
    from paper_1909_04631_gb300 import evaluate as ev
    prm = dict(scenes.STREET_PARAMS)
    scans = list(scenes.street_sequence(2, n_beams=16, n_az=384, first=4))
    p = sb.default_params(**prm, pool_blocks=1 << 15, sample_capacity=1 << 22, device=0, sensor_model=model)
    m = sb.Map(p)
    om = orc.OracleMap(orc.params(**dict(prm, sensor_model=model)))
    for sc in scans:
        m.insert_scan(sc["points"], sc["labels"], sc["pose"])
        om.insert_scan(sc["points"], sc["labels"], sc["pose"])
    K = prm["num_classes"]
    g = ev.map_quality(lambda x: m.query(x, var=False, mode=False, state=False), scans, K, prm["free_step"], 4)
    o = ev.map_quality(om.query, scans, K, prm["free_step"], 4)
    assert g["hits"] == o["hits"] and g["free_probes"] == o["free_probes"] > 0
    tol = 1e-5 if model == 1 else 2e-3
    np.testing.assert_allclose(np.nan_to_num(g["iou"], nan=-1), np.nan_to_num(o["iou"], nan=-1), atol=tol)
    assert abs(g["miou"] - o["miou"]) <= tol and abs(g["auc"] - o["auc"]) <= tol
    assert 0.0 < g["miou"] <= 1.0 and 0.5 < g["auc"] <= 1.0
