"""One map sharded over R ranks (one process per GPU), with one exchange step.

Every block of B^3 voxels has one owner rank, owner(block) = mix(block) mod R
(a fixed 64-bit mixing of the block coordinates).  After steps a1-a3 (each
rank turns its own scans into training points), every training point goes to
the owners of the blocks that hold a voxel centre within l of it (the
touched-block rule of step a4, Sec. IV); each rank then runs a4-a5 on what it
received.  A block's alpha is complete on its owner, since every point that
reaches it was routed there, so no reduction follows: the map is the union of
the owned blocks.  Blocks a rank touched but does not own hold partial sums
and are never read (export and queries keep owned blocks only).

The exchange uses point-to-point sends of torch.distributed (NCCL between GPUs,
gloo on the CPU).  The per-rank map is any object with the interface of
``Map``: ``insert_training(xyz, labels)``, ``export()`` and ``query(xyz)``.
"""
from __future__ import annotations

import numpy as np


def owner(blocks, world: int) -> np.ndarray:
    """Owner rank of each block (int64 [n,3] block coordinates)."""
    b = np.asarray(blocks, np.int64).reshape(-1, 3).astype(np.uint64)
    with np.errstate(over="ignore"):
        h = b[:, 0] * np.uint64(0x9E3779B97F4A7C15)
        h ^= b[:, 1] * np.uint64(0xC2B2AE3D27D4EB4F) + (h << np.uint64(6)) + (h >> np.uint64(2))
        h ^= b[:, 2] * np.uint64(0x165667B19E3779F9) + (h << np.uint64(6)) + (h >> np.uint64(2))
        h ^= h >> np.uint64(29)
        h *= np.uint64(0xBF58476D1CE4E5B9)
        h ^= h >> np.uint64(32)
    return (h % np.uint64(world)).astype(np.int64)


def touched_blocks(xyz, res: float, length_scale: float, block_edge: int):
    """For each point, the blocks of the 3x3x3 neighbourhood of its own block
    that hold a voxel centre strictly within l of it (FP64, the nearest centre
    of the block per axis; a relative margin of 1e-9 on l^2 keeps the set a
    superset of what the FP32/FP64 device test can reach).  Returns
    (point index [m], block [m,3])."""
    x = np.asarray(xyz, np.float64).reshape(-1, 3)
    B = int(block_edge)
    if length_scale > B * res:
        raise ValueError("length_scale reaches past the 3x3x3 block neighbourhood")
    v = np.floor(x.astype(np.float32) * np.float32(1.0 / res)).astype(np.int64)  # the voxel key of the point
    b0 = np.floor_divide(v, B)
    offs = np.stack(np.meshgrid(*([np.arange(-1, 2)] * 3), indexing="ij"), -1).reshape(-1, 3)
    blk = b0[:, None, :] + offs[None, :, :]                                   # [n,27,3]
    first, last = blk * B, blk * B + (B - 1)
    near = np.clip(np.rint(x[:, None, :] / res - 0.5), first, last)         # nearest voxel per axis
    e = (near + 0.5) * res - x[:, None, :]
    d2 = (e[..., 0] * e[..., 0] + e[..., 1] * e[..., 1]) + e[..., 2] * e[..., 2]
    # the rounded index may miss the nearest centre by one near a half-voxel tie: take the better of
    # it and its neighbours along each axis, all clamped into the block
    for ax in range(3):
        for step in (-1, 1):
            alt = near.copy()
            alt[..., ax] = np.clip(alt[..., ax] + step, first[..., ax], last[..., ax])
            ea = (alt + 0.5) * res - x[:, None, :]
            d2 = np.minimum(d2, (ea[..., 0] * ea[..., 0] + ea[..., 1] * ea[..., 1]) + ea[..., 2] * ea[..., 2])
    hit = d2 < length_scale * length_scale * (1.0 + 1e-9)
    pi, ki = np.nonzero(hit)
    return pi, blk[pi, ki]


def destinations(xyz, res: float, length_scale: float, block_edge: int, world: int):
    """(point index, rank) pairs: each point once for every rank owning a block it touches."""
    pi, blk = touched_blocks(xyz, res, length_scale, block_edge)
    pairs = np.unique(np.stack([pi, owner(blk, world)], 1), axis=0)
    return pairs[:, 0], pairs[:, 1]


def exchange(xyzl, dest_point, dest_rank, rank: int, world: int, device="cpu"):
    """Sends row dest_point[j] of xyzl [n,w] (float32; training points are
    x, y, z, label) to rank dest_rank[j] and returns every row this rank
    received, ordered by source rank and, within a source, by destination
    order, its own included, as a float32 tensor on `device` (the halo
    all-to-all; "cuda" tensors for the NCCL backend).  Counts go first (one
    all_gather), then one send/receive pair per peer."""
    import torch
    import torch.distributed as dist
    rows = np.asarray(xyzl, np.float32)
    if rows.ndim != 2:
        raise ValueError("rows must be a 2-D array")
    width = rows.shape[1]
    order = np.argsort(dest_rank, kind="stable")
    dp, dr = dest_point[order], dest_rank[order]
    counts = np.bincount(dr, minlength=world).astype(np.int64)
    starts = np.concatenate([[0], np.cumsum(counts)])
    outgoing = [torch.from_numpy(np.ascontiguousarray(rows[dp[starts[r]:starts[r + 1]]])).to(device)
                for r in range(world)]
    all_counts = [torch.zeros(world, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(all_counts, torch.from_numpy(counts).to(device))
    incoming = [torch.empty((int(all_counts[r][rank]), width), dtype=torch.float32, device=device)
                for r in range(world)]
    incoming[rank] = outgoing[rank]
    reqs = []
    for r in range(world):
        if r == rank:
            continue
        if outgoing[r].shape[0]:
            reqs.append(dist.isend(outgoing[r], dst=r))
        if incoming[r].shape[0]:
            reqs.append(dist.irecv(incoming[r], src=r))
    for q in reqs:
        q.wait()
    return torch.cat(incoming, 0)


class ShardedMap:
    """The part of one map that this rank owns; see the module docstring."""

    def __init__(self, local_map, res: float, length_scale: float, block_edge: int, rank: int, world: int,
                 device="cpu"):
        self.local = local_map
        self.device = device
        self.res, self.l, self.B = float(res), float(length_scale), int(block_edge)
        self.rank, self.world = int(rank), int(world)
        if self.l > self.B * self.res:
            raise ValueError("length_scale reaches past the 3x3x3 block neighbourhood")

    def insert_training(self, xyz, labels) -> int:
        """Routes this rank's training points to the owners of the blocks they
        touch and inserts what this rank receives; returns that count."""
        x = np.asarray(xyz, np.float32).reshape(-1, 3)
        lab = np.asarray(labels).reshape(-1)
        xyzl = np.concatenate([x, lab.astype(np.float32)[:, None]], 1)
        dp, dr = destinations(x, self.res, self.l, self.B, self.world)
        got = exchange(xyzl, dp, dr, self.rank, self.world, self.device)
        if got.shape[0]:
            if got.is_cuda:  # device buffers straight to the library
                import torch
                self.local.insert_training(got[:, :3].contiguous(), got[:, 3].to(torch.int32))
            else:
                g = got.numpy()
                self.local.insert_training(g[:, :3], g[:, 3].astype(np.int32))
        return int(got.shape[0])

    def owns_voxels(self, keys) -> np.ndarray:
        k = np.asarray(keys, np.int64).reshape(-1, 3)
        return owner(np.floor_divide(k, self.B), self.world) == self.rank

    def query(self, xyz, query_fields=("label", "p_occ")):
        """Read-off at this rank's world points: each point goes to the owner of
        its voxel's block, which answers from its map; every rank calls this
        together (collective).  Returns a dict of the query_fields, float64
        (labels as integers in float), in the order of xyz."""
        x = np.asarray(xyz, np.float32).reshape(-1, 3)
        dr = query_owner(x, self.res, self.B, self.world)
        dp = np.arange(len(x))
        tagged = np.concatenate([x, dp[:, None].astype(np.float32)], 1)  # exact below 2^24 points
        if len(x) >= (1 << 24):
            raise ValueError("at most 2^24 query points per call")
        got = exchange(tagged, dp, dr, self.rank, self.world).numpy()
        # the answers go back to where each point came from
        src_counts = self._source_counts(len(dp), dr)
        src = np.repeat(np.arange(self.world), src_counts)
        ans = self.local.query(got[:, :3]) if len(got) else {f: np.zeros(0) for f in query_fields}
        back = np.concatenate([got[:, 3:4]] + [np.asarray(ans[f], np.float64).reshape(-1, 1).astype(np.float32)
                                               for f in query_fields], 1)
        ret = exchange(back, np.arange(len(back)), src, self.rank, self.world).numpy()
        out = {}
        idx = ret[:, 0].astype(np.int64)
        for j, f in enumerate(query_fields):
            v = np.empty(len(x))
            v[idx] = ret[:, 1 + j]
            out[f] = v
        return out

    def _source_counts(self, n, dest_rank):
        """How many query points each rank sent to this one (one all_gather)."""
        import torch
        import torch.distributed as dist
        counts = torch.from_numpy(np.bincount(dest_rank, minlength=self.world).astype(np.int64))
        every = [torch.zeros(self.world, dtype=torch.int64) for _ in range(self.world)]
        dist.all_gather(every, counts)
        return np.array([int(e[self.rank]) for e in every], np.int64)

    def export(self):
        """(keys, alpha, pairs) of the voxels of the blocks this rank owns."""
        keys, alpha, pairs = self.local.export()[:3]
        keep = self.owns_voxels(keys)
        return keys[keep], alpha[keep], (pairs[keep] if pairs is not None else None)


def voxel_of(xyz, res: float) -> np.ndarray:
    """The voxel key floor(x * fp32(1/res)) of world points (the read-off's key)."""
    return np.floor(np.asarray(xyz, np.float32).reshape(-1, 3) * np.float32(1.0 / res)).astype(np.int64)


def query_owner(xyz, res: float, block_edge: int, world: int) -> np.ndarray:
    """The rank that answers a read-off query at each world point."""
    return owner(np.floor_divide(voxel_of(xyz, res), int(block_edge)), world)


__all__ = ["owner", "touched_blocks", "destinations", "exchange", "ShardedMap", "voxel_of", "query_owner"]
