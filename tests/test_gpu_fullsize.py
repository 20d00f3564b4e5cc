"""Parity at the sizes the benchmark runs.

- One whole 64 x 2048 LiDAR street scan (the benchmark's per-scan update):
  every voxel of the map against the FP64 oracle map, in both accumulation
  forms (keys and pair counts exact, alpha within relative 1e-5).
- The batched ingest at the benchmark's shape: 32 independent maps, one scan
  each, point counts log-uniform in 5k..250k, LiDAR- or depth-shaped.  Every
  map equals the map one sbki_insert_scan builds (keys and pairs exact, alpha
  to the order of FP32 reductions); the largest and the smallest maps equal
  the oracle's; a replay of the recorded graph adds exactly the same update
  again (pairs doubled, increments doubled).
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


# ------------------------------------------------------------ one whole street scan

@pytest.fixture(scope="module")
def street(orc):
    sc = next(scenes.street_sequence(1, first=7))
    prm = dict(scenes.STREET_PARAMS)
    om = orc.OracleMap(orc.params(**prm))
    ost = om.insert_scan(sc["points"], sc["labels"], sc["pose"])
    okeys, oalpha, opairs = om.export()
    return sc, prm, ost, okeys, oalpha, opairs


@pytest.mark.parametrize("mode", [0, 1], ids=["point_major", "block_major"])
def test_street_scan_whole_map(sb, street, mode):
    sc, prm, ost, okeys, oalpha, opairs = street
    p = sb.default_params(**prm, pool_blocks=1 << 16, sample_capacity=1 << 23, track_pairs=1, accumulate_mode=mode,
                          device=0)
    with sb.Map(p) as m:
        st = m.insert_scan(sc["points"], sc["labels"], sc["pose"])
        keys, alpha, pairs = m.export(pairs=True)
    assert st["train_points"] == ost["train"]
    assert keys.shape == okeys.shape and len(keys) > 2_000_000
    np.testing.assert_array_equal(keys, okeys)
    np.testing.assert_array_equal(pairs, opairs)
    assert st["pairs"] == int(opairs.sum())
    rel = _rel(alpha, oalpha)
    assert rel.max() <= RTOL, "max rel err %.3g" % rel.max()


# ------------------------------------------------------------ the batch at the benchmark's shape

PRM = dict(scenes.BATCH_PARAMS, num_classes=19)


@pytest.fixture(scope="module")
def batch():
    return scenes.batch_scans(n_maps=32)


def _params(sb, num_maps):
    return sb.default_params(**PRM, num_maps=num_maps, pool_blocks=1 << 18, sample_capacity=1 << 26, track_pairs=1,
                             device=0)


def _exports(m, n):
    out = []
    for i in range(n):
        m.select(i)
        out.append(m.export(pairs=True))
    return out


def test_batch_bench_shape_against_single_updates_oracle_and_replay(sb, orc, batch):
    import torch
    n = len(batch)
    sizes = np.array([len(s["points"]) for s in batch])
    assert n == 32 and sizes.min() >= 5000 and sizes.max() <= 250000
    dev = [dict(points=torch.from_numpy(s["points"]).cuda(), labels=torch.from_numpy(s["labels"]).cuda(),
                pose=s["pose"], map_id=i) for i, s in enumerate(batch)]
    with sb.Map(_params(sb, n)) as mb, sb.Map(_params(sb, n)) as ms:
        st = mb.insert_batch(dev)  # records the graph
        got = _exports(mb, n)
        pairs_single = 0
        for i, s in enumerate(batch):
            ms.select(i)
            pairs_single += ms.insert_scan(dev[i]["points"], dev[i]["labels"], s["pose"])["pairs"]
        ref = _exports(ms, n)
        assert st["pairs"] == pairs_single
        for i in range(n):
            (k, a, p), (rk, ra, rp) = got[i], ref[i]
            np.testing.assert_array_equal(k, rk)
            np.testing.assert_array_equal(p, rp)
            assert _rel(a, ra).max(initial=0.0) <= RTOL, i  # FP32 reductions in another order
        # the oracle for the largest and the smallest maps
        order = np.argsort(sizes)
        for i in list(order[-2:]) + list(order[:1]):
            om = orc.OracleMap(orc.params(**PRM))
            om.insert_scan(batch[i]["points"], batch[i]["labels"], batch[i]["pose"])
            ok, oa, op = om.export()
            k, a, p = got[i]
            np.testing.assert_array_equal(k, ok)
            np.testing.assert_array_equal(p, op)
            assert _rel(a, oa).max() <= RTOL, (i, _rel(a, oa).max())
        # a replay of the recording adds the same update again
        st2 = mb.insert_batch(dev)
        assert st2["pairs"] == st["pairs"]
        again = _exports(mb, n)
        a0 = np.float64(PRM["alpha0"])
        for i in range(n):
            (k, a, p), (k2, a2, p2) = got[i], again[i]
            np.testing.assert_array_equal(k2, k)
            np.testing.assert_array_equal(p2, 2 * p)
            inc, inc2 = a.astype(np.float64) - a0, a2.astype(np.float64) - a0
            touched = p > 0
            np.testing.assert_allclose(inc2[touched], 2 * inc[touched], rtol=1e-5, atol=1e-9)


# ------------------------------------------------------------ the differentiable form at full size

def _world(points, pose):
    """world = fp32(((r0 px + r1 py) + r2 pz) + t) in FP64 (the transform reading)."""
    T = np.asarray(pose, np.float64).reshape(4, 4)
    p = np.asarray(points, np.float32).astype(np.float64)
    out = np.empty((len(p), 3), np.float32)
    for a in range(3):
        out[:, a] = (((T[a, 0] * p[:, 0] + T[a, 1] * p[:, 1]) + T[a, 2] * p[:, 2]) + T[a, 3]).astype(np.float32)
    return out


def _oracle_slab(args):
    """The oracle's held-out log-likelihood and gradient for the held-out points
    of one slab, given every training point that can reach their voxels."""
    prm, idx, x64, lab, hx, hl = args
    from oracle import oracle as O
    ll, gl, gs, gx = O.heldout_grad(O.params(**prm), x64, lab, hx, hl)
    return ll, gl, gs, idx, gx


def _oracle_grad_parallel(prm, xyz, lab, held, held_lab, slabs):
    """LL and its gradient are sums over held-out points, and a held-out point
    sees alpha only at its own voxel, i.e. only training points within l + res
    of it (in x).  So the oracle runs per slab of held-out points (in x) with
    the training points of the slab widened by that margin, in parallel
    processes, and the slabs' terms are added up."""
    import multiprocessing as mp
    import os
    margin = prm["length_scale"] + prm["res"]
    edges = np.quantile(held[:, 0], np.linspace(0.0, 1.0, slabs + 1))
    edges[-1] = np.inf
    x64 = xyz.astype(np.float64)
    jobs = []
    for s in range(slabs):
        hs = (held[:, 0] >= edges[s]) & (held[:, 0] < edges[s + 1]) if s > 0 else held[:, 0] < edges[1]
        if not hs.any():
            continue
        lo, hi = held[hs, 0].min() - margin, held[hs, 0].max() + margin
        ts = np.nonzero((xyz[:, 0] >= lo) & (xyz[:, 0] <= hi))[0]
        jobs.append((prm, ts, x64[ts], lab[ts], held[hs], held_lab[hs]))
    assert sum(len(j[4]) for j in jobs) == len(held)
    with mp.get_context("spawn").Pool(min(slabs, os.cpu_count() or 1)) as pool:
        parts = pool.map(_oracle_slab, jobs, chunksize=1)
    ll = sum(p[0] for p in parts)
    gl = sum(p[1] for p in parts)
    gs = sum(p[2] for p in parts)
    gx = np.zeros_like(x64)
    for p in parts:
        np.add.at(gx, p[3], p[4])
    return ll, gl, gs, gx


def test_differentiable_form_full_size(sb):
    """20 LiDAR scans (64 x 2048) of the small region, 20 % of the hits held out:
    LL (relative 1e-5), dLL/dl and dLL/dsigma0 (relative 1e-4) over all ~8M
    training points, and dLL/dxyz at 4096 seeded occupied training points
    (the error's norm within 1e-4 of the gradient's norm there) against the
    FP64 oracle."""
    prm = dict(scenes.DIFF_PARAMS)
    scans = list(scenes.small_region_lidar_sequence(20))
    p = sb.default_params(**prm, pool_blocks=1 << 16, sample_capacity=1 << 23, device=0)
    xs, ls = [], []
    with sb.Map(p) as m:
        for sc in scans:
            x, l = m.training_set(sc["points"], sc["labels"], sc["pose"])
            xs.append(x)
            ls.append(l)
    xyz = np.concatenate(xs)
    lab = np.concatenate(ls).astype(np.int32)
    held = np.concatenate([_world(sc["held_points"], sc["pose"]) for sc in scans])
    held_lab = np.concatenate([sc["held_labels"] for sc in scans]).astype(np.int32)
    assert len(xyz) > 7_000_000 and len(held) > 400_000
    xyzl = np.concatenate([xyz, lab[:, None].astype(np.float32)], 1)
    with sb.Map(p) as m:
        m.insert_training(xyz, lab)
        m.grad_clear()
        ll = m.heldout_loglik(held, held_lab, grad=True)
        gl, gs, gx = m.backward(xyzl)
    oll, ogl, ogs, ogx = _oracle_grad_parallel(prm, xyz, lab, held, held_lab, slabs=32)
    assert abs(ll - oll) <= 1e-5 * abs(oll), (ll, oll)
    assert abs(gl - ogl) <= 1e-4 * abs(ogl), (gl, ogl)
    assert abs(gs - ogs) <= 1e-4 * abs(ogs), (gs, ogs)
    rng = np.random.default_rng(3)
    pick = rng.choice(np.nonzero(lab >= 1)[0], size=4096, replace=False)
    err = np.abs(gx[pick].astype(np.float64) - ogx[pick])
    assert np.linalg.norm(err) <= 1e-4 * np.linalg.norm(ogx[pick])
    assert np.all(err <= 1e-3 * np.abs(ogx[pick]) + 1e-5 * np.abs(ogx[pick]).max())
