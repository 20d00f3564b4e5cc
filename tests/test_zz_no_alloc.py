"""The training-set entry point that allocates nothing (sbki_training_set_noalloc).

Callers that cannot allocate device memory while they run (a real-time loop
that reserves everything at start-up, a framework that owns the device heap)
use it.  It must give the same training set as sbki_training_set on the same
scan, bit for bit (the training-set tolerance of the parity tests), on
consecutive calls that share its fixed device array, leave the device's free
memory unchanged, and reject inputs beyond its limits without disturbing
later calls.  Collected last so that it also runs after every other GPU test
in the same process.
"""
import numpy as np
import pytest

from synth import scenes

pytestmark = pytest.mark.gpu

MAX_POINTS = 16384


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
    prm.update(kw)
    return sb.default_params(res=prm["res"], length_scale=prm["length_scale"], sigma0=prm["sigma0"],
                             alpha0=prm["alpha0"], free_step=prm["free_step"], num_classes=prm["num_classes"],
                             min_range=prm["min_range"], max_range=prm["max_range"], pool_blocks=1 << 12,
                             sample_capacity=1 << 21, device=0)


def _sorted(xyzl):
    order = np.lexsort((xyzl[:, 3], xyzl[:, 2], xyzl[:, 1], xyzl[:, 0]))
    return xyzl[order]


def _noalloc(sb, p, pts, lab, pose, cap, out=None, check_free=False):
    """One call on inputs and output allocated beforehand; with check_free, the
    device's free memory must be the same before and after the call."""
    import torch
    dp = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    dl = torch.from_numpy(np.ascontiguousarray(lab, np.int32)).cuda()
    if out is None:
        out = torch.full((cap, 4), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n = sb.training_set_noalloc(p, dp, dl, pose, out)
    torch.cuda.synchronize()
    if check_free:
        assert torch.cuda.mem_get_info()[0] == free0, "free device memory changed during the call"
    return out[:n].cpu().numpy(), n


def _reference(sb, p, pts, lab, pose):
    with sb.Map(p) as m:
        x, l = m.training_set(pts, lab, pose)
    return np.concatenate([x, l.astype(np.float32)[:, None]], 1)


def test_noalloc_matches_training_set_on_consecutive_calls(sb):
    p = _params(sb)
    # a larger scan, then a smaller one: the second call must not see the first's leftovers
    cases = [(scenes.small_region_scan(0), 3500), (scenes.small_region_scan(1), 2000)]
    for k, (sc, n) in enumerate(cases):
        pts, lab = sc["points"][:n], sc["labels"][:n]
        # from the second call on, the device set-up is done: nothing may be allocated
        got, cnt = _noalloc(sb, p, pts, lab, sc["pose"], cap=1 << 17, check_free=k > 0)
        ref = _reference(sb, p, pts, lab, sc["pose"])
        assert cnt == len(ref) > 0
        np.testing.assert_array_equal(_sorted(got), _sorted(ref))


def test_noalloc_limits_then_recovers(sb):
    p = _params(sb)
    sc = scenes.small_region_scan(2)
    T = sc["pose"]
    # more input points than the fixed array holds: rejected before any GPU work
    big = np.zeros((MAX_POINTS + 1, 3), np.float32)
    with pytest.raises(sb.SbkiError) as e:
        _noalloc(sb, p, big, np.ones(MAX_POINTS + 1, np.int32), T, cap=16)
    assert e.value.status == sb.ERR_INVALID_ARG
    # a full scan has ~290k hits + free samples, beyond the 131072 the array holds
    with pytest.raises(sb.SbkiError) as e:
        _noalloc(sb, p, sc["points"], sc["labels"], T, cap=16)
    assert e.value.status == sb.ERR_CAPACITY
    # output capacity too small: cap points written, the full count reported by the error
    import torch
    n = 1200
    ref = _reference(sb, p, sc["points"][:n], sc["labels"][:n], T)
    small = torch.full((64, 4), float("nan"), dtype=torch.float32, device="cuda")
    with pytest.raises(sb.SbkiError) as e:
        _noalloc(sb, p, sc["points"][:n], sc["labels"][:n], T, cap=64, out=small)
    assert e.value.status == sb.ERR_CAPACITY
    assert e.value.count == len(ref)
    written = small.cpu().numpy()
    ref_rows = {tuple(r) for r in ref.view(np.uint32).tolist()}
    assert all(tuple(r) in ref_rows for r in written.view(np.uint32).tolist()), "rows outside the training set"
    assert len({tuple(r) for r in written.view(np.uint32).tolist()}) == 64
    # the shared array's leftovers from the failed calls do not leak into the next one
    got, cnt = _noalloc(sb, p, sc["points"][:n], sc["labels"][:n], T, cap=1 << 17, check_free=True)
    assert cnt == len(ref)
    np.testing.assert_array_equal(_sorted(got), _sorted(ref))
