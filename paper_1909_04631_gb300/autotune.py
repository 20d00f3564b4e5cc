"""Autotuner of the update's launch shapes.

The kernels of the update run on persistent grids whose shapes (CTAs per SM
of the accumulation, training points per warp chunk, CTAs per SM of the
touched-block pass and of the ingest kernels) change speed, not results; so
does the form of the accumulation (point-major or block-major: the same keys
and pair counts, alpha up to the order of FP32 sums).  `autotune` times
candidate shapes and forms on scratch handles built from the caller's
parameters, fed the caller's batch of scans through `sbki_insert_batch` (one
warm-up call, which also records the batch's CUDA graph, then `reps` timed
calls with CUDA events), and returns the fastest, with the time of the
library's default shape beside it.  The block edge is not swept: it changes
which voxels a map allocates.  Results can be kept in a JSON cache keyed by
device, geometry and batch shape.  Everything it times runs in libsbki's
kernels; this module only chooses and records shapes.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

from . import sbki as _sb

DEFAULT_CANDIDATES = dict(accumulate_ctas_per_sm=(0, 2, 3), accumulate_chunk=(4, 10, 20, 30),
                          touch_ctas_per_sm=(4, 8), ingest_ctas_per_sm=(8, 16))


def split_tuning(tuning):
    """(launch shapes for Map.set_tuning, accumulate_mode or None) of a tuning dict."""
    t = dict(tuning)
    return t, t.pop("accumulate_mode", None)


def _key(params, scans, device_name):
    geo = [params.res, params.length_scale, params.free_step, params.ds_res, params.max_range, params.num_classes,
           params.block_edge, params.accumulate_mode, params.sensor_model]
    shape = [len(scans), int(sum(len(s["points"]) for s in scans) // 10000)]
    return hashlib.sha1(json.dumps([device_name, geo, shape]).encode()).hexdigest()[:16]


def autotune(params, scans, candidates=None, reps=3, cache_path=None, stream=None):
    """Best launch shapes for updates like `scans` (a batch as for Map.insert_batch).

    Returns dict(tuning=..., ms=..., trials=[(tuning, ms), ...], default_ms=..., cached=bool);
    tuning holds the launch shapes (for Map.set_tuning) and accumulate_mode
    (a map parameter: split it off with split_tuning)."""
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
    # the block-major form takes neither the counting model nor per-class length scales
    one_form = params.sensor_model != 0 or any(params.l_scale[k] != 1.0 for k in range(params.num_classes + 1))
    modes = tuple(cand.pop("accumulate_mode", (int(params.accumulate_mode),) if one_form else (0, 1)))
    names = list(cand)
    stream = stream if stream is not None else torch.cuda.current_stream(dev)
    trials = []

    def timed(m):
        m.insert_batch(scans)  # warm-up, records the graph for this shape
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            m.insert_batch(scans)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    default_ms = None
    for mode in modes:
        q = _sb.Params.from_buffer_copy(params)
        q.accumulate_mode = mode
        with _sb.Map(q, stream=stream) as m:
            default = m.get_tuning()
            if mode == int(params.accumulate_mode):
                default_ms = timed(m)  # the library's own shape, untuned
            for values in itertools.product(*(cand[n] for n in names)):
                t = dict(zip(names, values))
                m.set_tuning(**t)
                trials.append((dict(t, accumulate_mode=mode), timed(m)))
            m.set_tuning(**default)
    best, ms = min(trials, key=lambda x: x[1])
    result = dict(tuning=best, ms=ms, trials=trials, default_ms=default_ms)
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as fh:
                cache = json.load(fh)
        cache[key] = dict(tuning=best, ms=ms, trials=trials, default_ms=default_ms)
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as fh:
            json.dump(cache, fh)
    return dict(result, cached=False)
