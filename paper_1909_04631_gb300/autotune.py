"""Autotuner of the update's launch shapes.

The kernels of the update run on persistent grids whose shapes (CTAs per SM
of the accumulation, training points per warp chunk, CTAs per SM of the
touched-block pass and of the ingest kernels) change speed, not results.
`autotune` times candidate shapes on a scratch handle built from the caller's
parameters, fed the caller's batch of scans through `sbki_insert_batch` (one
warm-up call, which also records the batch's CUDA graph, then `reps` timed
calls with CUDA events), and returns the fastest.  Results can be kept in a
JSON cache keyed by device, geometry and batch shape.  Everything it times
runs in libsbki's kernels; this module only chooses and records shapes.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

from . import sbki as _sb

DEFAULT_CANDIDATES = dict(accumulate_ctas_per_sm=(0, 2, 3), accumulate_chunk=(4, 10, 20, 30),
                          touch_ctas_per_sm=(4, 8), ingest_ctas_per_sm=(8, 16))


def _key(params, scans, device_name):
    geo = [params.res, params.length_scale, params.free_step, params.ds_res, params.max_range, params.num_classes,
           params.block_edge, params.accumulate_mode, params.sensor_model]
    shape = [len(scans), int(sum(len(s["points"]) for s in scans) // 10000)]
    return hashlib.sha1(json.dumps([device_name, geo, shape]).encode()).hexdigest()[:16]


def autotune(params, scans, candidates=None, reps=3, cache_path=None, stream=None):
    """Best launch shapes for updates like `scans` (a batch as for Map.insert_batch).

    Returns dict(tuning=..., ms=..., trials=[(tuning, ms), ...], cached=bool)."""
    import torch
    dev = torch.device("cuda", params.device)
    name = torch.cuda.get_device_name(dev)
    key = _key(params, scans, name)
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
        if key in cache:
            return dict(cache[key], cached=True)
    cand = dict(DEFAULT_CANDIDATES, **(candidates or {}))
    names = list(cand)
    stream = stream if stream is not None else torch.cuda.current_stream(dev)
    trials = []
    with _sb.Map(params, stream=stream) as m:
        for values in itertools.product(*(cand[n] for n in names)):
            t = dict(zip(names, values))
            m.set_tuning(**t)
            m.insert_batch(scans)  # warm-up, records the graph for this shape
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                m.insert_batch(scans)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            trials.append((t, e0.elapsed_time(e1) / reps))
    best, ms = min(trials, key=lambda x: x[1])
    result = dict(tuning=best, ms=ms, trials=trials)
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as fh:
                cache = json.load(fh)
        cache[key] = dict(tuning=best, ms=ms, trials=trials)
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as fh:
            json.dump(cache, fh)
    return dict(result, cached=False)
