"""The tile autotuner's host logic with fake timings: it keeps the fastest
candidate and caches it as JSON keyed by GPU name and batch signature (the
per-problem shapes and the format table); a cached entry is reused without
timing, and force re-times."""
import json

from paper_2310_07854_gb300 import autotune
from paper_2310_07854_gb300 import formats as F
from paper_2310_07854_gb300 import synth


def test_cache_keyed_by_gpu_and_batch(tmp_path, monkeypatch):
    import torch
    probs = synth.make_uneven_problems(n_problems=3)
    fake = {32: 2.0, 64: 1.5, 128: 1.0, 256: 1.2}
    timed = []

    def time_tile(problems, table, tile, reps=7):
        timed.append(tile)
        return fake[tile]

    monkeypatch.setattr(autotune, "time_tile", time_tile)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "GPU-A")
    cache = str(tmp_path / "tiles.json")
    r = autotune.tune(probs, F.FP32_TABLE, cache_path=cache)
    assert r["tile"] == 128 and not r["cached"] and sorted(timed) == [32, 64, 128, 256]
    timed.clear()
    r = autotune.tune(probs, F.FP32_TABLE, cache_path=cache)
    assert r["cached"] and r["tile"] == 128 and timed == []
    # another format table, another batch: new keys
    assert not autotune.tune(probs, F.FormatTable.parse("G=E2M1"), cache_path=cache)["cached"]
    assert not autotune.tune(probs[:2], F.FP32_TABLE, cache_path=cache)["cached"]
    # another GPU: its own entry
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "GPU-B")
    fake[64] = 0.5
    r = autotune.tune(probs, F.FP32_TABLE, cache_path=cache)
    assert not r["cached"] and r["tile"] == 64
    # force re-times even when cached
    timed.clear()
    assert not autotune.tune(probs, F.FP32_TABLE, cache_path=cache, force=True)["cached"]
    assert len(timed) == len(autotune.CANDIDATES)
    data = json.load(open(cache))
    assert set(data) == {"GPU-A", "GPU-B"} and len(data["GPU-A"]) == 3
    assert data["GPU-A"][autotune.signature(probs, F.FP32_TABLE)]["tile"] == 128
