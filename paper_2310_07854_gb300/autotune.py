"""Tile-size autotuner for the uneven-batch launch.

For a batch it times one captured CUDA-graph replay of vapr_batched_eval
per candidate tile (median of several replays, CUDA events) and keeps the
fastest.  Results persist in a JSON cache keyed by GPU name and a signature
of the batch (per-problem configurations, cuboids, spheres, self pairs and
the format table), so a shape is tuned once.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

from . import formats as F

CANDIDATES = (32, 64, 128, 256)


def default_cache_path() -> str:
    return os.environ.get("VAPR_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "vapr_gb300", "tiles.json"))


def signature(problems, table: F.FormatTable) -> str:
    h = hashlib.sha256()
    for w in problems:
        h.update(f"{w.n},{w.scene.n_cuboids},{w.robot.n_spheres},{w.robot.n_pairs};".encode())
    h.update(str(table).encode())
    return h.hexdigest()[:24]


def time_tile(problems, table, tile: int, reps: int = 7) -> float:
    """Median ms of one graph replay of the batch at this tile."""
    import torch
    from .batched import BatchedEvaluator
    ev = BatchedEvaluator(problems, table, tile=tile)
    g = ev.capture()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def tune(problems, table: F.FormatTable = F.FP32_TABLE, candidates=CANDIDATES,
         cache_path: str | None = None, force: bool = False) -> dict:
    """-> {"tile": best, "ms": {tile: median ms}, "cached": bool}."""
    import torch
    cache_path = cache_path or default_cache_path()
    gpu = torch.cuda.get_device_name()
    sig = signature(problems, table)
    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    ent = cache.get(gpu, {}).get(sig)
    if ent and not force:
        return {**ent, "cached": True}
    ms = {t: time_tile(problems, table, t) for t in candidates}
    best = min(ms, key=ms.get)
    ent = {"tile": best, "ms": {str(k): v for k, v in ms.items()}}
    cache.setdefault(gpu, {})[sig] = ent
    os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, cache_path)
    return {**ent, "cached": False}
