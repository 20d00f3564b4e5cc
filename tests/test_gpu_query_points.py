"""Eq. (alpha_kernel) at arbitrary query points (sbki_query_points) against the
oracle's all-pairs FP64 sum (alpha_at_points, pinned on the CPU): alpha within
relative 1e-5 at arbitrary points, at voxel centres equal to the map update's
alpha (the same sum in another FP32 order), host and device buffers, empty
inputs, and a whole street scan's training set."""
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


@pytest.mark.parametrize("seed,l,K", [(0, 0.3, 4), (1, 0.15, 11), (2, 0.45, 2)])
def test_query_points_match_oracle(sb, orc, seed, l, K):
    rng = np.random.default_rng(seed)
    n = 3000
    xyz = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    xyz[: n // 10] = (np.round(xyz[: n // 10] / 0.1) * 0.1).astype(np.float32)
    lab = rng.integers(0, K + 1, size=n).astype(np.int32)
    prm = dict(res=0.1, length_scale=l, sigma0=0.37, alpha0=0.001, num_classes=K)
    p = sb.default_params(**prm, device=0)
    q = np.concatenate([rng.uniform(-1.2, 1.2, size=(1500, 3)),  # arbitrary points
                        xyz[:200] + rng.normal(0, 0.02, size=(200, 3)),  # next to training points
                        xyz[200:260],  # on training points
                        [[40.0, 40.0, 40.0], [-9.0, 3.0, 1.0]]]).astype(np.float32)  # far away: the prior
    xyzl = np.concatenate([xyz, lab[:, None].astype(np.float32)], 1)
    got = sb.query_points(p, xyzl, q)
    want = orc.alpha_at_points(orc.params(**prm), xyz, lab, q.astype(np.float64))
    assert _rel(got, want).max() <= RTOL
    assert np.all(got[-2:] == np.float32(0.001))
    # device buffers, written in place
    import torch
    out = torch.empty((len(q), K + 1), dtype=torch.float32, device="cuda")
    sb.query_points(p, torch.from_numpy(xyzl).cuda(), torch.from_numpy(q).cuda(), out=out)
    np.testing.assert_array_equal(out.cpu().numpy(), got)


def test_query_points_at_voxel_centres_equal_the_map(sb):
    rng = np.random.default_rng(7)
    xyz = rng.uniform(-0.8, 0.8, size=(2500, 3)).astype(np.float32)
    lab = rng.integers(0, 6, size=2500).astype(np.int32)
    prm = dict(res=0.1, length_scale=0.3, sigma0=0.5, alpha0=0.001, num_classes=5)
    p = sb.default_params(**prm, pool_blocks=1 << 12, sample_capacity=1 << 20, device=0)
    sb.set_param(p, "sigma0_scale", [0.7, 1.3, 1.0, 2.0, 0.5, 1.1])
    with sb.Map(p) as m:
        m.insert_training(xyz, lab)
        keys, alpha, _ = m.export()
    centres = ((keys + 0.5) * 0.1).astype(np.float32)
    xyzl = np.concatenate([xyz, lab[:, None].astype(np.float32)], 1)
    got = sb.query_points(p, xyzl, centres)
    # the centres as FP32 are not the FP64 centres of the map, so compare where that cannot matter
    assert _rel(got, alpha).max() <= 2e-5


def test_query_points_empty_inputs(sb):
    p = sb.default_params(res=0.1, length_scale=0.3, num_classes=3, device=0)
    q = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 3.0]], np.float32)
    got = sb.query_points(p, np.zeros((0, 4), np.float32), q)
    assert np.all(got == np.float32(p.alpha0))
    assert sb.query_points(p, np.zeros((0, 4), np.float32), np.zeros((0, 3), np.float32)).shape == (0, 4)
    bad = sb.default_params(res=0.1, length_scale=0.3, num_classes=3, sensor_model=1, device=0)
    with pytest.raises(sb.SbkiError) as e:
        sb.query_points(bad, np.zeros((1, 4), np.float32), q)
    assert e.value.status == sb.ERR_INVALID_ARG


def test_query_points_street_training_set(sb, orc):
    """A whole 64 x 2048 street scan's training set (~720k points) queried at
    2000 seeded points near its hits against the oracle's all-pairs sum."""
    sc = next(scenes.street_sequence(1, first=5))
    prm = dict(scenes.STREET_PARAMS)
    p = sb.default_params(**prm, pool_blocks=1 << 16, sample_capacity=1 << 23, device=0)
    with sb.Map(p) as m:
        x, lab = m.training_set(sc["points"], sc["labels"], sc["pose"])
    rng = np.random.default_rng(11)
    pick = rng.choice(len(x), size=2000, replace=False)
    q = (x[pick] + rng.normal(0, 0.05, size=(2000, 3))).astype(np.float32)
    xyzl = np.concatenate([x, lab[:, None].astype(np.float32)], 1)
    got = sb.query_points(p, xyzl, q)
    want = orc.alpha_at_points(orc.params(**prm), x, lab, q.astype(np.float64))
    assert _rel(got, want).max() <= RTOL
