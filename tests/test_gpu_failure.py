"""Failure detection without a GPU fault: a device-side wait whose flag is never
set (the look-back of one radix-sort digit pass, over tiles whose first one is
never processed) runs out after its bound and reports SBKI_ERR_TIMEOUT; the
context stays usable."""
import time

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


def test_bounded_wait_reports_timeout_and_context_survives(sb):
    t0 = time.time()
    assert sb.sbki.selftest_bounded_wait(0) == sb.ERR_TIMEOUT
    assert time.time() - t0 < 30.0
    # the device still works: a small update gives the usual result
    pts, lab = scenes.random_cloud(2000, 7, extent=1.0, num_classes=3)
    p = sb.default_params(res=0.1, length_scale=0.3, sigma0=1.0, num_classes=3, pool_blocks=1 << 12,
                          sample_capacity=1 << 20, device=0)
    with sb.Map(p) as m:
        st = m.insert_training(pts, lab)
        assert st["pairs"] > 0
        keys, alpha, _ = m.export()
        assert np.all(np.isfinite(alpha)) and keys.shape[0] > 0
