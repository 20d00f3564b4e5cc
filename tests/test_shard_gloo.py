"""One map sharded over ranks (host logic of the multi-GPU design) without a
GPU: the halo rule against the oracle's touched blocks, block ownership, and
two gloo ranks whose owned blocks together equal the single map built from
all their training points.  The oracle stands in for each rank's map."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp

from paper_1909_04631_gb300 import shard

PRM = dict(res=0.1, length_scale=0.3, sigma0=0.7, alpha0=0.001, num_classes=4, block_edge=8)


def _cloud(seed, n):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-1.3, 1.5, size=(n, 3))
    xyz[: n // 5] = np.round(xyz[: n // 5] / 0.8) * 0.8 + rng.uniform(-0.31, 0.31, size=(n // 5, 3))  # near block faces
    return xyz.astype(np.float32), rng.integers(0, 5, size=n).astype(np.int32)


def test_halo_rule_equals_oracle_touched_blocks(orc):
    """touched_blocks of each point = the blocks the oracle allocates for that point alone (Eq. alpha_kernel)."""
    xyz, lab = _cloud(41, 60)
    pi, blk = shard.touched_blocks(xyz, PRM["res"], PRM["length_scale"], PRM["block_edge"])
    for i in range(len(xyz)):
        m = orc.OracleMap(orc.params(**PRM))
        m.insert_training(xyz[i:i + 1], lab[i:i + 1])
        want = {tuple(k) for k in m.block_keys()}
        got = {tuple(b) for b in blk[pi == i]}
        assert got == want, i


def test_owner_is_a_balanced_function_of_the_block():
    rng = np.random.default_rng(2)
    blocks = rng.integers(-5000, 5000, size=(40000, 3))
    o = shard.owner(blocks, 4)
    np.testing.assert_array_equal(o, shard.owner(blocks.copy(), 4))
    counts = np.bincount(o, minlength=4)
    assert counts.min() > 0.22 * len(blocks)
    assert np.all(shard.owner(blocks, 1) == 0)
    with pytest.raises(ValueError):
        shard.touched_blocks(np.zeros((1, 3)), 0.1, 0.9, 8)


def _queries():
    rng = np.random.default_rng(47)
    return rng.uniform(-1.5, 1.7, size=(500, 3)).astype(np.float32)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    from oracle import oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        xyz, lab = _cloud(43, 900)
        mine = slice(rank, None, world)  # each rank ingests its own share of the points
        sm = shard.ShardedMap(orc.OracleMap(orc.params(**PRM)), PRM["res"], PRM["length_scale"], PRM["block_edge"],
                              rank, world)
        received = sm.insert_training(xyz[mine], lab[mine])
        keys, alpha, pairs = sm.export()
        # read-off at this rank's own query points, answered by the owners (rank 1 asks nothing)
        q = _queries() if rank == 0 else np.zeros((0, 3), np.float32)
        ans = sm.query(q)
        parts = [None] * world
        dist.all_gather_object(parts, (keys, alpha, pairs, received, ans))
        out[rank] = parts if rank == 0 else None
    finally:
        dist.destroy_process_group()


def test_two_ranks_own_the_single_map(orc):
    ctx = tmp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        parts = out[0]
    keys = np.concatenate([p[0] for p in parts])
    alpha = np.concatenate([p[1] for p in parts])
    pairs = np.concatenate([p[2] for p in parts])
    assert all(p[3] > 0 for p in parts)
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    keys, alpha, pairs = keys[order], alpha[order], pairs[order]
    xyz, lab = _cloud(43, 900)
    single = orc.OracleMap(orc.params(**PRM))
    single.insert_training(xyz, lab)
    skeys, salpha, spairs = single.export()
    np.testing.assert_array_equal(keys, skeys)      # every block owned exactly once
    np.testing.assert_array_equal(pairs, spairs)
    np.testing.assert_allclose(alpha, salpha, rtol=1e-12)  # FP64 sums in another order
    # routed queries: the owners' answers equal the single map's read-off
    ans = parts[0][4]
    want = single.query(_queries())
    np.testing.assert_array_equal(ans["label"], want["label"])
    np.testing.assert_allclose(ans["p_occ"], want["p_occ"].astype(np.float32), rtol=1e-6)
    assert len(parts[1][4]["label"]) == 0
