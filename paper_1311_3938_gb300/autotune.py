"""Autotuner for batched stepping: tile bits, threads per CTA and PEC steps per graph replay.

For a sample of jobs it builds one batch per candidate shape, replays a fixed number of rounds
after one warm-up round, times them with CUDA events on the batch stream and keeps the shape
with the most amplitude-steps per second (sum over members of advanced steps x 2^n).  Results
are cached in a JSON file keyed by GPU name, precision and the sample's n-histogram.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import _native as N
from .engine import Batch
from .workloads import make_context

DEFAULT_SHAPES = [
    # (tile_bits, threads, steps_per_round)
    (0, 256, 16),
    (0, 256, 64),
    (0, 128, 16),
    (11, 256, 16),
    (12, 256, 16),
]


def _cache_path():
    base = os.environ.get("AQC_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "aqc_gb300")
    os.makedirs(base, exist_ok=True)
    return os.path.join(base, "autotune.json")


def _key(jobs, precision):
    name = torch.cuda.get_device_name()
    hist = {}
    for j in jobs:
        hist[j.n] = hist.get(j.n, 0) + 1
    return f"{name}|p{precision}|" + ",".join(f"{k}:{hist[k]}" for k in sorted(hist))


def measure_shape(jobs, shape, device=0, rounds=4):
    """Amplitude-steps per second of one batch shape on `jobs` (a short run, not to T)."""
    tile_bits, threads, spr = shape
    items = sum(1 << max(0, j.n - 5) for j in jobs) + 1024
    b = Batch(jobs[0].precision, device=device, max_members=len(jobs), max_items=items, threads=threads,
              steps_per_round=spr)
    ctxs = []
    try:
        for j in jobs:
            ctx, _ = make_context(j, device, tile_bits=tile_bits)
            b.add(ctx)
            ctxs.append(ctx)
        b.run(1)  # warm-up (builds and instantiates the graph)
        s0, _, _ = b.poll()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.run(rounds)
        e1.record(b.stream)
        s1, _, _ = b.poll()
        ms = e0.elapsed_time(e1)
        amp_steps = sum((s1[k] - s0[k]) * (1 << ctxs[k].n) for k in range(len(ctxs)) if s1[k] >= 0)
        return amp_steps / (ms * 1e-3) if ms > 0 else 0.0
    finally:
        b.close()
        for c in ctxs:
            c.close()


def autotune(jobs, shapes=None, device=0, use_cache=True, rounds=4):
    """Best (tile_bits, threads, steps_per_round) for batches like `jobs`."""
    shapes = shapes or DEFAULT_SHAPES
    key = _key(jobs, jobs[0].precision)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except Exception:
            cache = {}
        if key in cache:
            return tuple(cache[key]["shape"]), cache[key]
    results = []
    for sh in shapes:
        t0 = time.perf_counter()
        rate = measure_shape(jobs, sh, device, rounds)
        results.append({"shape": list(sh), "amp_steps_per_s": rate, "wall_s": time.perf_counter() - t0})
    best = max(results, key=lambda r: r["amp_steps_per_s"])
    entry = {"shape": best["shape"], "results": results}
    if use_cache:
        cache[key] = entry
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return tuple(best["shape"]), entry
