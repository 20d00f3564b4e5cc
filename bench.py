#!/usr/bin/env python3
"""Benchmark of the S-BKI per-scan map update on one GB300 (or N replicas).

Workload: the LiDAR street sequence (64 x 2048 beams over +2 to -24.8 deg,
max range 50 m, 19 occupied classes + free, 0.1 m voxels, l = 0.3 m, free
samples every 0.3 m, sigma0 = 0.1, alpha0 = 0.001), synthetic and seeded.
A step is one whole scan update through the C ABI (transform, free-space
sampling, downsampling, block hash, kernel accumulation) into a map that
persists over the sequence; scans are resident in HBM before timing.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on bounded samples of the same scans (azimuth sectors) instead.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import scenes  # noqa: E402

METRIC = "LiDAR scans/sec (64x2048 street sequence, S-BKI per-scan update)"
# roofline model of one in-support pair of Eq. (kernel) as the paper writes it:
# ~14 FP32 operations and 3 MUFU operations (sqrt, sin, cos); per SM and clock
# 128 FP32 lanes and 16 MUFU lanes
PAIR_CLK_PER_SM = max(14.0 / 128.0, 3.0 / 16.0)
# sources of the accumulation kernel (a committed DRAM-traffic figure is valid only for these bytes)
KERNEL_SOURCES = ["paper_1909_04631_gb300/csrc/accumulate_points.cu", "paper_1909_04631_gb300/csrc/kernel_value.cuh",
                  "paper_1909_04631_gb300/csrc/kernel_poly.cuh", "paper_1909_04631_gb300/csrc/point_common.cuh"]


def _gen(args):
    first, count = args
    return [dict(points=s["points"], labels=s["labels"], clean_labels=s["clean_labels"], pose=s["pose"])
            for s in scenes.street_sequence(count, first=first)]


def generate_scans(first, count, workers):
    """Scans first..first+count-1, generated on the host with a spawn pool."""
    if count <= 0:
        return []
    chunks = []
    per = max(1, math.ceil(count / max(1, workers)))
    for a in range(first, first + count, per):
        chunks.append((a, min(per, first + count - a)))
    if workers <= 1 or len(chunks) == 1:
        out = []
        for c in chunks:
            out += _gen(c)
        return out
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(workers, len(chunks))) as pool:
        parts = pool.map(_gen, chunks)
    return [s for p in parts for s in p]


def sector(scan, k, nsec):
    """Points of scan in azimuth sector k of nsec (sensor frame)."""
    p = scan["points"]
    az = np.arctan2(p[:, 1], p[:, 0])
    s = np.floor((az + np.pi) / (2 * np.pi) * nsec).astype(int) % nsec
    sel = s == k
    return p[sel], scan["labels"][sel]


def oracle_rate(scans, n_steps, nsec=8, progress=None):
    """FP64 oracle on azimuth sectors: step i processes sector i % nsec of
    scan i // nsec into one persistent map.  Returns (scans/s, pairs/s,
    seconds, steps)."""
    from oracle import oracle as O
    p = O.params(**scenes.STREET_PARAMS)
    m = O.OracleMap(p)
    t_total = 0.0
    for i in range(n_steps):
        sc = scans[(i // nsec) % len(scans)]
        pts, lab = sector(sc, i % nsec, nsec)
        t0 = time.perf_counter()
        m.insert_scan(pts, lab, sc["pose"])
        t_total += time.perf_counter() - t0
    _, _, pc = m.export()
    if t_total <= 0.0:
        return 0.0, 0.0, 0.0
    return (n_steps / nsec) / t_total, float(pc.sum()) / t_total, t_total


# --- the oracle on all host cores: one process per core, each with its own map,
# sectors handed out by a pool (the oracle itself unchanged and single-threaded)
_OW = {}


def _orc_worker_init(scans, nsec):
    from oracle import oracle as O
    _OW["scans"], _OW["nsec"] = scans, nsec
    _OW["map"] = O.OracleMap(O.params(**scenes.STREET_PARAMS))


def _orc_worker_task(job):
    si, k = job
    sc = _OW["scans"][si]
    pts, lab = sector(sc, k, _OW["nsec"])
    t0 = time.perf_counter()
    _OW["map"].insert_scan(pts, lab, sc["pose"])
    return time.perf_counter() - t0


class OraclePool:
    """workers processes on the host cores (spawned before any GPU call), each
    inserting whole azimuth sectors into its own oracle map."""

    def __init__(self, scans, workers, nsec=8):
        from oracle import oracle as O
        O.build()
        self.nsec, self.n, self.next = nsec, len(scans), 0
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_orc_worker_init, initargs=(scans, nsec))
        # every worker started and its oracle loaded before any timing
        self.pool.map(_orc_worker_task, [(0, 0)] * workers, chunksize=1)

    def run(self, n_sectors):
        """Wall seconds for the next n_sectors sectors, spread over the workers."""
        jobs = []
        for _ in range(n_sectors):
            i = self.next
            self.next += 1
            jobs.append(((i // self.nsec) % self.n, i % self.nsec))
        t0 = time.perf_counter()
        list(self.pool.imap_unordered(_orc_worker_task, jobs, chunksize=1))
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region, into a
    temporary file (or the path given)."""

    def __init__(self, index=0, path=None):
        import tempfile
        self.index = index
        self.proc = None
        self.path = path or os.path.join(tempfile.mkdtemp(prefix="sbki_clocks_"), "clocks.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        # the sampler is running once its first line is out; only later lines count
        self.skip = 0
        t_end = time.time() + 5.0
        while self.proc is not None and time.time() < t_end and self.proc.poll() is None:
            self.fh.flush()
            n = sum(1 for _ in open(self.path))
            if n > 0:
                self.skip = n
                break
            time.sleep(0.01)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in list(open(self.path))[self.skip:]:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[2:]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def profiled_traffic():
    """DRAM bytes per launch of the accumulation kernel from the committed ncu
    summary, or None when the kernel sources changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "accumulate_points_lidar_street.txt")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    if fields.get("sources_sha256") != h.hexdigest() or "dram_bytes_per_launch" not in fields:
        return None
    return float(fields["dram_bytes_per_launch"])


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


def replica_first_scan(rank):
    """Replicas only: rank r maps its own stretch of street, scans from 1000 r on."""
    return rank * 1000


def max_over_ranks(value, world, device):
    """The slowest rank's figure (every rank returns it)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _gen_batch(n_maps):
    return scenes.batch_scans(n_maps=n_maps)


def _gen_diff(n_scans):
    return list(scenes.small_region_lidar_sequence(n_scans))


def _gen_single():
    return scenes.small_region_scan(0)


def _gen_depth(n_frames):
    return list(scenes.room_sequence(n_frames))


def other_workloads(sb, torch, dev, stream, single, frames):
    """The single-scan workload (fresh map per update) and the depth-camera
    sequence (one map), device inputs, CUDA events."""
    out = {}
    p = sb.default_params(**scenes.SMALL_SCENE_PARAMS, pool_blocks=1 << 14, sample_capacity=1 << 22,
                          device=dev.index)
    pts, lab = torch.from_numpy(single["points"]).to(dev), torch.from_numpy(single["labels"]).to(dev)
    maps = [sb.Map(p, stream=stream) for _ in range(12)]
    times, st = [], None
    for k, m in enumerate(maps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = m.insert_scan(pts, lab, single["pose"])
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            times.append(e0.elapsed_time(e1))
        m.close()
    ms = float(np.median(times))
    out["single_scan"] = {"workload": "one 100x100-ray scan of the 20x20x4 m region into a fresh map",
                          "hits": st["hits"], "pairs": st["pairs"], "ms_per_scan": ms, "scans_per_s": 1e3 / ms,
                          "pairs_per_s": st["pairs"] / (ms / 1e3)}
    q = sb.default_params(**scenes.ROOM_PARAMS, pool_blocks=1 << 17, sample_capacity=1 << 24, device=dev.index)
    dp = [torch.from_numpy(f["points"]).to(dev) for f in frames]
    dl = [torch.from_numpy(f["labels"]).to(dev) for f in frames]
    with sb.Map(q, stream=stream) as m:
        for i in range(2):
            m.insert_scan(dp[i], dl[i], frames[i]["pose"])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pairs = 0
        for i in range(2, len(frames)):
            pairs += m.insert_scan(dp[i], dl[i], frames[i]["pose"])["pairs"]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (len(frames) - 2)
    out["depth_camera"] = {"workload": "640x480 depth frames of the room sequence (0.05 m voxels, l = 0.15 m, 11 classes)",
                           "frames": len(frames) - 2, "ms_per_frame": ms, "frames_per_s": 1e3 / ms,
                           "pairs_per_s": pairs / (len(frames) - 2) / (ms / 1e3)}
    return out


def batched_form(sb, torch, dev, stream, scans, reps):
    """Independent maps, one scan each: one batched update (recorded graph)
    against one sbki_insert_scan per scan, on the same GPU (device inputs)."""
    prm = dict(scenes.BATCH_PARAMS, num_classes=19)
    n = len(scans)
    total = sum(len(s["points"]) for s in scans)
    p = sb.default_params(**prm, num_maps=n, pool_blocks=1 << 18, sample_capacity=1 << 26, device=dev.index)
    dp = [torch.from_numpy(s["points"]).to(dev) for s in scans]
    dl = [torch.from_numpy(s["labels"]).to(dev) for s in scans]
    batch = [dict(points=dp[i], labels=dl[i], pose=scans[i]["pose"], map_id=i) for i in range(n)]

    def timed(fn):
        fn()  # warm-up (and the graph recording of the batched form)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    from paper_1909_04631_gb300 import autotune
    tuned = autotune.autotune(p, batch, reps=2, stream=stream)
    shapes, mode = autotune.split_tuning(tuned["tuning"])
    if mode is not None:
        p.accumulate_mode = mode
    seq = sb.Map(p, stream=stream)
    seq.set_tuning(**shapes)

    def run_seq():
        for i in range(n):
            seq.select(i)
            seq.insert_scan(dp[i], dl[i], scans[i]["pose"])

    ms_seq = timed(run_seq)
    seq.close()
    bat = sb.Map(p, stream=stream)
    bat.set_tuning(**shapes)
    st = {}

    def run_batch():
        st.update(bat.insert_batch(batch))

    ms_batch = timed(run_batch)
    launches = bat.profile_read()["launches"]
    bat.close()
    return {"workload": "%d independent maps, one scan each: N log-uniform 5k..250k, LiDAR- or depth-shaped, "
                        "0.1 m voxels, l = 0.3 m" % n, "scans": n, "points": total,
            "train_points": st.get("train_points"), "pairs": st.get("pairs"), "reps": reps,
            "sequential_ms": ms_seq, "batched_ms": ms_batch, "sequential_scans_per_s": n / (ms_seq / 1e3),
            "batched_scans_per_s": n / (ms_batch / 1e3), "speedup": ms_seq / ms_batch,
            "batched_kernels_per_update": launches // (reps + 1), "tuning": tuned["tuning"],
            "tuning_trials": len(tuned["trials"]), "untuned_batched_ms": tuned.get("default_ms")}


def differentiable_form(sb, torch, dev, stream, scans, reps):
    """Held-out log-likelihood and its gradient w.r.t. l, sigma0 and every
    training point on the small-region LiDAR sequence, against forward only."""
    prm = dict(scenes.DIFF_PARAMS)
    p = sb.default_params(**prm, pool_blocks=1 << 16, sample_capacity=1 << 23, device=dev.index)
    xs, ls, hx, hl = [], [], [], []
    with sb.Map(p, stream=stream) as m:
        for sc in scans:
            x, l = m.training_set(sc["points"], sc["labels"], sc["pose"])
            xs.append(x)
            ls.append(l)
            T = np.asarray(sc["pose"], np.float64).reshape(4, 4)
            hp = sc["held_points"].astype(np.float64)
            hw = np.stack([(((T[a, 0] * hp[:, 0] + T[a, 1] * hp[:, 1]) + T[a, 2] * hp[:, 2]) + T[a, 3])
                           for a in range(3)], 1).astype(np.float32)
            hx.append(hw)
            hl.append(sc["held_labels"])
    xyz = torch.from_numpy(np.concatenate(xs)).to(dev)
    lab = torch.from_numpy(np.concatenate(ls).astype(np.int32)).to(dev)
    xyzl = torch.cat([xyz, lab[:, None].float()], 1).contiguous()
    held = torch.from_numpy(np.concatenate(hx)).to(dev)
    held_lab = torch.from_numpy(np.concatenate(hl).astype(np.int32)).to(dev)
    maps = [sb.Map(p, stream=stream) for _ in range(2 * reps + 2)]
    res = {}
    for mode in ("forward", "forward_backward"):
        times = []
        for r in range(reps + 1):
            m = maps.pop()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            m.insert_training(xyz, lab)
            if mode == "forward":
                ll = m.heldout_loglik(held, held_lab)
            else:
                m.grad_clear()
                ll = m.heldout_loglik(held, held_lab, grad=True)
                gl, gs, gx = m.backward(xyzl)
            e1.record(stream)
            torch.cuda.synchronize()
            if r > 0:
                times.append(e0.elapsed_time(e1))
            m.close()
        res[mode + "_ms"] = float(np.median(times))
    for m in maps:
        m.close()
    return {"workload": "%d LiDAR scans (64x2048) of the 20x20x4 m region, 20%% of hits held out; gradient w.r.t. "
                        "l, sigma0 and all %d training points" % (len(scans), xyz.shape[0]),
            "train_points": int(xyz.shape[0]), "held_out": int(held.shape[0]), "reps": reps, **res,
            "backward_overhead": res["forward_backward_ms"] / res["forward_ms"]}


def run_reference(args, rank, world):
    """The FP64 oracle on all host cores: each step inserts one azimuth sector
    (1/8 scan) per core, the cores working in parallel into maps of their own."""
    if rank != 0:
        return 0
    scans = generate_scans(0, 2, args.workers)
    cores = host_cores()
    nsec = 8
    pool = OraclePool(scans, cores, nsec)
    if args.warmup > 0:
        pool.run(args.warmup * cores)
    secs = pool.run(args.steps * cores)
    pool.close()
    rate = args.steps * cores / nsec / secs
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "scans/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded street scene, ray-cast)",
            "config": {"workload": "lidar-street-64x2048", "beams": 64, "azimuths": 2048, "classes": 19,
                       "res_m": 0.1, "length_scale_m": 0.3, "free_step_m": 0.3},
            "cpu_baseline": {"value": rate, "unit": "scans/s", "cores": cores, "kind": "oracle",
                             "sample": "each step = one 45-degree azimuth sector (1/8 scan of 64x2048) per host "
                                       "core, %d cores in parallel (one process and map each); scans/s = "
                                       "sectors / 8 / wall seconds" % cores},
            "e2e": {"value": rate, "unit": "scans/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def counting_model(sb, torch, stream, p, dpts, dlab, poses, warmup, steps):
    """The street sequence through the counting sensor model (Eq. alpha): the
    same ingest, then one count per training point in the voxel holding it.
    Device inputs, CUDA events; stage times from the library's own events."""
    nscan = len(dpts)
    with sb.Map(p, stream=stream, sensor_model=1) as m:
        for i in range(warmup):
            m.insert_scan(dpts[i % nscan], dlab[i % nscan], poses[i % nscan])
        m.profile(True, reset=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        e0.record(stream)
        for i in range(steps):
            j = (warmup + i) % nscan
            stats.append(m.insert_scan(dpts[j], dlab[j], poses[j]))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = m.profile_read()
    n = max(1, prof["inserts"])
    K1 = scenes.STREET_PARAMS["num_classes"] + 1
    train = sum(s["train_points"] for s in stats) / steps
    newb = sum(s["new_blocks"] for s in stats) / steps
    # algorithmic bytes of the count step per scan: the training point (16 B), its
    # hash slot (key + pool index, 12 B) and the read-modify-write of one alpha
    # word (8 B) per point, and the zero fill of the blocks created by the scan
    acc_s = prof["accumulate_ms"] / 1e3 / n
    bytes_alg = 36.0 * train + 4.0 * K1 * 512 * newb
    bw, _, src = peaks()
    return {"workload": "LiDAR street 64x2048 sequence, counting sensor model (Eq. alpha), 0.1 m voxels",
            "scans": steps, "ms_per_scan": ms, "scans_per_s": 1e3 / ms, "train_points_per_scan": train,
            "stage_ms": {"ingest": prof["ingest_ms"] / n, "blocks": prof["blocks_ms"] / n,
                         "count": prof["accumulate_ms"] / n},
            "count_step": {"bytes_alg": bytes_alg, "achieved_gbs": bytes_alg / acc_s / 1e9, "peak_gbs": bw,
                           "frac": bytes_alg / acc_s / 1e9 / bw, "peak_source": "hbm_gbs of %s peaks" % src}}


def _street_probs(labels, K, seed):
    """Seeded softmax vectors over classes 1..K, peaked (logit + 3) at each hit's label."""
    rng = np.random.default_rng(seed)
    lab = np.clip(np.asarray(labels), 1, K) - 1
    logits = rng.normal(0.0, 1.0, size=(len(lab), K)).astype(np.float32)
    logits[np.arange(len(lab)), lab] += np.float32(3.0)
    e = np.exp(logits - logits.max(1, keepdims=True))
    return (e / e.sum(1, keepdims=True)).astype(np.float32)


def street_forms(sb, torch, stream, p, scans, dpts, dlab, poses, warmup, steps):
    """The street sequence under the map's other rules: soft labels (a softmax
    vector over the 19 classes per hit), the extended-block association (a
    voxel takes the points of its block and the six face neighbours) and
    per-class length scales.  Device inputs, CUDA events around the updates,
    stage times from the library's own events.  The soft-label entry point
    synchronises its stream once per call (it sizes the soft buffers)."""
    K = scenes.STREET_PARAMS["num_classes"]
    nscan = len(dpts)
    steps = min(steps, 20)
    used = sorted({i % nscan for i in range(warmup + steps)})
    probs = {j: torch.from_numpy(_street_probs(scans[j]["labels"], K, 500 + j)).to(dpts[j].device) for j in used}
    rng = np.random.default_rng(9)
    lscale = [1.0] + [float(v) for v in rng.uniform(0.7, 1.3, size=K)]

    def timed(m, insert):
        for i in range(warmup):
            insert(m, i % nscan)
        m.profile(True, reset=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = [insert(m, (warmup + i) % nscan) for i in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = m.profile_read()
        n = max(1, prof["inserts"])
        return {"scans": steps, "ms_per_scan": ms, "scans_per_s": 1e3 / ms,
                "pairs_per_scan": sum(x["pairs"] for x in st) / steps,
                "train_points_per_scan": sum(x["train_points"] for x in st) / steps,
                "stage_ms": {"ingest": prof["ingest_ms"] / n, "blocks": prof["blocks_ms"] / n,
                             "accumulate": prof["accumulate_ms"] / n}}

    hard = lambda m, j: m.insert_scan(dpts[j], dlab[j], poses[j])  # noqa: E731
    out = {}
    with sb.Map(p, stream=stream) as m:
        out["soft_labels"] = dict(timed(m, lambda m, j: m.insert_scan_soft(dpts[j], probs[j], poses[j])),
                                  input="softmax over 19 classes per hit (seeded logits N(0,1), +3 at the label)")
    with sb.Map(p, stream=stream, association=1) as m:
        out["extended_block"] = timed(m, hard)
    with sb.Map(p, stream=stream, l_scale=lscale) as m:
        out["per_class_length_scale"] = dict(timed(m, hard), l_scale=lscale)
    return out


def map_quality_form(sb, stream, p, scans, n=20):
    """Both sensor models on the first n street scans, scored on those scans
    against the generator's clean labels (before the label noise): IoU of the
    map's labels at the hits and AUC of p_occ, hits against points the beams
    passed through (every 16th beam).  Not timed."""
    from paper_1909_04631_gb300 import evaluate as ev
    out = {"workload": "street scans 0..%d inserted, then scored on their own hits and beams" % (n - 1),
           "ground_truth": "clean labels of the generator (before the 10 % label noise)"}
    K = scenes.STREET_PARAMS["num_classes"]
    for name, model in (("s_bki", 0), ("s_csm", 1)):
        with sb.Map(p, stream=stream, sensor_model=model) as m:
            for sc in scans[:n]:
                m.insert_scan(sc["points"], sc["labels"], sc["pose"])
            q = ev.map_quality(lambda x: m.query(x, var=False, mode=False, state=False), scans[:n], K,
                               scenes.STREET_PARAMS["free_step"], stride=16)
        fin = lambda v: None if v != v else v  # noqa: E731  (NaN: a class neither present nor predicted)
        out[name] = {"miou": fin(q["miou"]), "auc": fin(q["auc"]), "iou": [fin(round(v, 4)) for v in q["iou"]]}
        out["hits"], out["free_probes"] = q["hits"], q["free_probes"]
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1909_04631_gb300 as sb

    # host-side generation before any GPU call (spawn pool)
    nscan = min(args.scans, args.warmup + args.steps)
    scans = generate_scans(replica_first_scan(rank), nscan, args.workers)
    forms_input = None
    if rank == 0 and not args.no_forms:
        ctx = mp.get_context("spawn")
        with ctx.Pool(4) as pool:
            fb = pool.apply_async(_gen_batch, (32,))
            fd = pool.apply_async(_gen_diff, (20,))
            fs = pool.apply_async(_gen_single)
            fr = pool.apply_async(_gen_depth, (12,))
            forms_input = (fb.get(), fd.get(), fs.get(), fr.get())
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on bounded samples, before any GPU call: all host cores (one
        # process and map per core, 8 azimuth sectors of 45 degrees each, about
        # 7 s), then one core (12 sectors: scan 0 whole, half of scan 1, about 10 s)
        cores = host_cores()
        pool = OraclePool(scans[:2], cores, 8)
        secs_all = pool.run(8 * cores)
        pool.close()
        rate, prate, secs = oracle_rate(scans[:2], 12, 8)
        depth = None
        if forms_input is not None:  # one ray in eight of a 640x480 depth frame of the room sequence, one core
            from oracle import oracle as O
            fr = forms_input[3][0]
            om = O.OracleMap(O.params(**scenes.ROOM_PARAMS))
            t0 = time.perf_counter()
            om.insert_scan(fr["points"][::8], fr["labels"][::8], fr["pose"])
            dt = time.perf_counter() - t0
            depth = {"value": 1.0 / (8.0 * dt), "unit": "frames/s", "cores": 1,
                     "sample": "one ray in eight of a 640x480 depth frame (room sequence, 0.05 m voxels); "
                               "frames/s = 1 / (8 x %.2f s)" % dt}
        cpu = {"value": cores / secs_all, "unit": "scans/s", "cores": cores, "kind": "oracle",
               "sample": "%d azimuth sectors of 45 deg (sectors of scans 0 and 1 of 64x2048, cycled), FP64, "
                         "%d host cores in parallel (one process and map each); scans/s = %d / %.2f s"
                         % (8 * cores, cores, cores, secs_all),
               "one_core": {"value": rate, "cores": 1, "pairs_per_s": prate,
                            "sample": "12 azimuth sectors of 45 deg (scan 0, half of scan 1) into one map; "
                                      "scans/s = 1.5 / %.2f s" % secs},
               "one_core_depth": depth}

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    stream = torch.cuda.current_stream(dev)
    p = sb.default_params(**{k: v for k, v in scenes.STREET_PARAMS.items()}, pool_blocks=args.pool_blocks,
                          sample_capacity=args.sample_capacity, device=local_rank)
    m = sb.Map(p, stream=stream)
    dpts = [torch.from_numpy(s["points"]).to(dev) for s in scans]
    dlab = [torch.from_numpy(s["labels"]).to(dev) for s in scans]
    poses = [s["pose"] for s in scans]
    torch.cuda.synchronize()

    for i in range(args.warmup):
        j = i % nscan
        m.insert_scan(dpts[j], dlab[j], poses[j])
    m.profile(True, reset=True)
    launches0 = m.profile_read()["launches"]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # scans streamed through the asynchronous entry point: each update still reads its
    # counters back once (to size the sort), but the host issues the next scan without
    # waiting for the end of the previous one; errors surface at the sync below
    with ClockSampler(local_rank, args.clock_log) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            j = (args.warmup + i) % nscan
            m.insert_scan(dpts[j], dlab[j], poses[j], sync=False)
        ev1.record(stream)
        torch.cuda.synchronize()
    m.sync()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    prof = m.profile_read()
    launches = prof["launches"] - launches0
    m.profile(False, reset=True)

    m.close()
    # end to end through the C ABI from pinned host buffers (H2D inside the call,
    # stats D2H): a fresh map fed the same warm-up and timed scans
    hp = [torch.from_numpy(s["points"]).pin_memory() for s in scans]
    hl = [torch.from_numpy(s["labels"]).pin_memory() for s in scans]
    m = sb.Map(p, stream=stream)
    for i in range(args.warmup):
        j = i % nscan
        m.insert_scan(hp[j].numpy(), hl[j].numpy(), poses[j])
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = 0
    for i in range(args.steps):
        j = (args.warmup + i) % nscan
        m.insert_scan(hp[j].numpy(), hl[j].numpy(), poses[j], sync=False)
        h2d += hp[j].numel() * 4 + hl[j].numel() * 4
    last = m.sync()  # the stats of the last update (device to host)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    d2h = prof["readback_bytes"] + 80 // args.steps  # the counters once per update; the final stats once
    m.close()

    if rank != 0:
        return 0
    # per-scan counts (untimed): the same scans in the same order into a fresh map, one synchronous update each
    # and each such update timed on its own (CUDA events around it): the per-scan latency
    stats, lat = [], []
    with sb.Map(p, stream=stream) as sm:
        for i in range(args.warmup + args.steps):
            j = i % nscan
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record(stream)
            s = sm.insert_scan(dpts[j], dlab[j], poses[j])
            q1.record(stream)
            if i >= args.warmup:
                stats.append(s)
                q1.synchronize()
                lat.append(q0.elapsed_time(q1))
    assert stats[-1]["pairs"] == last["pairs"] and stats[-1]["train_points"] == last["train_points"]
    # voxels touched per scan (untimed): the block-major form counts them; the
    # same scans in the same order into a fresh map give the same touched sets
    acc = sb.Map(p, stream=stream, accumulate_mode=1)
    acc_stats = []
    for i in range(args.warmup + args.steps):
        j = i % nscan
        if i == args.warmup:
            acc.profile(True, reset=True)
        s = acc.insert_scan(dpts[j], dlab[j], poses[j])
        if i >= args.warmup:
            acc_stats.append(s)
    acc_prof = acc.profile_read()
    acc.close()
    assert [s["pairs"] for s in acc_stats] == [s["pairs"] for s in stats], "block-major pass saw other pairs"
    K1 = scenes.STREET_PARAMS["num_classes"] + 1
    B3 = 512
    pairs = sum(s["pairs"] for s in stats)
    vt = sum(s["touched_voxels"] for s in acc_stats)
    newb = sum(s["new_blocks"] for s in stats)
    # algorithmic work of the accumulation step per scan (one fresh-fill and one
    # accumulation launch): read+write alpha[K+1] of each touched voxel and the
    # zero-fill of new blocks; pair arithmetic of Eq. (kernel) per in-support pair
    bytes_alg = (8.0 * K1 * vt + 4.0 * K1 * B3 * newb) / args.steps
    pairs_per = pairs / args.steps
    acc_s = prof["accumulate_ms"] / 1e3 / max(1, prof["inserts"])
    bw, sm_mhz_max, src = peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    t_hbm = bytes_alg / (bw * 1e9)
    t_alu = pairs_per * PAIR_CLK_PER_SM / (n_sm * sm_mhz_max * 1e6)
    traffic = profiled_traffic()
    common = {"kernel": "accumulate_points_fast_kernel (+ fresh_fill_kernel)", "seconds_per_launch": acc_s,
              "bytes_alg_per_launch": bytes_alg, "pairs_per_launch": pairs_per, "touched_voxels_per_launch": vt / args.steps,
              "t_hbm_s": t_hbm, "t_alu_s": t_alu, "traffic": traffic}
    if t_alu > t_hbm:
        peak = n_sm * sm_mhz_max * 1e6 / PAIR_CLK_PER_SM / 1e9
        roof = {"bound": "alu", "achieved": pairs_per / acc_s / 1e9, "peak": peak, "unit": "Gpair/s",
                "frac": (pairs_per / acc_s / 1e9) / peak,
                "peak_source": "%d SMs x %.0f MHz / %.4f clk per pair (3 MUFU per pair)"
                               % (n_sm, sm_mhz_max, PAIR_CLK_PER_SM)}
    else:
        roof = {"bound": "hbm", "achieved": bytes_alg / acc_s / 1e9, "peak": bw, "unit": "GB/s",
                "frac": (bytes_alg / acc_s / 1e9) / bw, "peak_source": "hbm_gbs of %s peaks" % src}
    roof.update(common)
    value = args.steps * world / (ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "scans/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded street scene, ray-cast)",
        "config": {"workload": "lidar-street-64x2048", "beams": 64, "azimuths": 2048, "classes": 19,
                   "res_m": 0.1, "length_scale_m": 0.3, "free_step_m": 0.3, "distinct_scans": nscan,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "not flushed: each step touches %.0f MB of alpha blocks (> 129 MB L2)"
                         % (sum(s["touched_blocks"] for s in stats) / args.steps * K1 * B3 * 4 / 1e6)},
        "pairs_per_s": pairs * world / (ms / 1e3),
        "per_scan": {"hits": stats[-1]["hits"], "free_samples": stats[-1]["free_samples"],
                     "train_points": stats[-1]["train_points"], "pairs": int(pairs_per),
                     "touched_blocks": stats[-1]["touched_blocks"], "touched_voxels": int(vt / args.steps)},
        "stage_ms": {"ingest": prof["ingest_ms"] / max(1, prof["inserts"]),
                     "blocks": prof["blocks_ms"] / max(1, prof["inserts"]),
                     "accumulate": prof["accumulate_ms"] / max(1, prof["inserts"])},
        "roofline": roof,
        "per_scan_ms": {"median": float(np.median(lat)), "p90": float(np.percentile(lat, 90)),
                        "source": "%d synchronous sbki_insert_scan calls, CUDA events around each" % len(lat)},
        "accumulate_forms_ms": {"point_major": prof["accumulate_ms"] / max(1, prof["inserts"]),
                                "block_major": acc_prof["accumulate_ms"] / max(1, acc_prof["inserts"])},
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "e2e": {"value": args.steps * world / e2e_s, "unit": "scans/s",
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h,
                "api": "Map.insert_scan(host arrays, sync=False) per scan (sbki_insert_scan_async), Map.sync() at the end"},
        "cpu_baseline": cpu,
    }
    if forms_input is not None:
        line["batched"] = batched_form(sb, torch, dev, stream, forms_input[0], reps=5)
        line["differentiable"] = differentiable_form(sb, torch, dev, stream, forms_input[1], reps=3)
        line["other_workloads"] = other_workloads(sb, torch, dev, stream, forms_input[2], forms_input[3])
        line["counting_model"] = counting_model(sb, torch, stream, p, dpts, dlab, poses, args.warmup, args.steps)
        line["map_quality"] = map_quality_form(sb, stream, p, scans, n=min(20, len(scans)))
        line["street_forms"] = street_forms(sb, torch, stream, p, scans, dpts, dlab, poses, args.warmup, args.steps)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=97)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scans", type=int, default=100, help="distinct scans of the sequence to cycle over")
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and differentiable measurements")
    ap.add_argument("--pool-blocks", type=int, default=1 << 18, help="map block pool capacity")
    ap.add_argument("--sample-capacity", type=int, default=1 << 23, help="hits + free samples per scan")
    ap.add_argument("--clock-log", default=None, help="file for the nvidia-smi clock samples (default: a temp file)")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("need --steps >= 1 and --warmup >= 0")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
