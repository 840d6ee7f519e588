"""Autotuner of the batched persistent kernels' tile shape.

For a batch it times ``jxf_batch_step`` over a few steps for every candidate
(face-tile length x persistent blocks per SM, plus one-block-per-tile),
keeps the fastest and caches it in a JSON file keyed by the batch's
signature (precision, model, dimension, sorted grid sizes, device name).
Timing advances the batch's states: reset them afterwards.
"""
from __future__ import annotations

import hashlib
import json
import os

TILE_FACES = (256, 512, 1024, 2048, 4096, 8192)
BLOCKS_PER_SM = (0, 4, 8, 16)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "jxf_autotune.json")


def signature(batch) -> str:
    import torch
    sizes = sorted(tuple(c["n"]) for c in batch.cases)
    key = json.dumps([batch.precision, batch.cases[0]["model"], batch.cases[0]["ndim"], sizes,
                      torch.cuda.get_device_name()])
    return hashlib.sha1(key.encode()).hexdigest()


def tune(batch, steps: int = 3, cache: str = DEFAULT_CACHE, force: bool = False):
    """Pick (tile_faces, blocks_per_sm) for the batch, apply it and return
    (choice, {candidate: ms per step})."""
    import torch
    sig = signature(batch)
    table = {}
    if os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if not force and sig in table:
        tf, bps = table[sig]["choice"]
        batch.set_tiling(tf, bps)
        return (tf, bps), table[sig]["timings"]
    timings = {}
    for tf in TILE_FACES:
        for bps in BLOCKS_PER_SM:
            batch.set_tiling(tf, bps)
            batch.step(steps)  # builds the n-step graph and warms up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            batch.step(steps)
            e1.record()
            torch.cuda.synchronize()
            timings["%d,%d" % (tf, bps)] = e0.elapsed_time(e1) / steps
    best = min(timings, key=timings.get)
    tf, bps = (int(x) for x in best.split(","))
    batch.set_tiling(tf, bps)
    table[sig] = {"choice": [tf, bps], "timings": timings}
    os.makedirs(os.path.dirname(cache) or ".", exist_ok=True)
    tmp = cache + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, cache)
    return (tf, bps), timings
