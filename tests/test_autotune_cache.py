"""Host logic of the tile-shape cache (paper_1605_01800_gb300/autotune.py),
on the CPU: the library calls and the GPU name are replaced by fakes, so
only the keying, the reuse and the invalidation of cache entries run."""
import json
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1605_01800_gb300 import autotune, lbm  # noqa: E402

SHAPES = [(32, 16), (32, 8), (64, 8)]


class Fake:
    def __init__(self, monkeypatch, best=1, gpu="GPU-A"):
        self.tuned = 0
        self.selected = []
        self.best = best
        monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
        monkeypatch.setattr(torch.cuda, "get_device_name", lambda i=0: self.gpu)
        monkeypatch.setattr(lbm, "lbm_tile_count", lambda: len(SHAPES))
        monkeypatch.setattr(lbm, "lbm_tile_shape", lambda i: SHAPES[i])
        monkeypatch.setattr(lbm, "lbm_set_tile", lambda ctx, i: self.selected.append(i))
        monkeypatch.setattr(lbm, "lbm_autotune", self.autotune)
        self.gpu = gpu

    def autotune(self, ctx, steps):
        self.tuned += 1
        self.selected.append(self.best)
        return self.best, [1.0] * len(SHAPES)


def batch(sizes, precision=lbm.LBM_FP32_DEV, walls=False):
    specs = [types.SimpleNamespace(nx=nx, ny=ny, solid=np.zeros((ny, nx), np.uint8) if walls else None, eos="cs")
             for nx, ny in sizes]
    return types.SimpleNamespace(specs=specs, precision=precision, ctx=object())


def test_measures_once_then_reuses(monkeypatch, tmp_path):
    f = Fake(monkeypatch, best=2)
    cache = str(tmp_path / "tiles.json")
    r1 = autotune.best_tile(batch([(256, 64)] * 4), cache_path=cache)
    r2 = autotune.best_tile(batch([(256, 64)] * 4), cache_path=cache)
    assert (r1["tile"], r1["cached"], r2["tile"], r2["cached"]) == (2, False, 2, True)
    assert f.tuned == 1 and f.selected == [2, 2]
    stored = json.load(open(cache))
    assert list(stored.values()) == [{"tile": 2, "shape": [64, 8]}]


def test_key_covers_gpu_precision_and_lattices(monkeypatch, tmp_path):
    f = Fake(monkeypatch)
    cache = str(tmp_path / "tiles.json")
    autotune.best_tile(batch([(256, 64)]), cache_path=cache)
    autotune.best_tile(batch([(256, 64)], precision=lbm.LBM_FP64), cache_path=cache)
    autotune.best_tile(batch([(256, 64)], walls=True), cache_path=cache)
    autotune.best_tile(batch([(128, 64)]), cache_path=cache)
    f.gpu = "GPU-B"
    autotune.best_tile(batch([(256, 64)]), cache_path=cache)
    assert f.tuned == 5 and len(json.load(open(cache))) == 5
    # the order of the lattices in the batch does not matter
    f.gpu = "GPU-A"
    autotune.best_tile(batch([(64, 32), (256, 64)]), cache_path=cache)
    r = autotune.best_tile(batch([(256, 64), (64, 32)]), cache_path=cache)
    assert r["cached"] and f.tuned == 6


def test_stale_entries_are_measured_again(monkeypatch, tmp_path):
    f = Fake(monkeypatch, best=1)
    cache = str(tmp_path / "tiles.json")
    b = batch([(256, 64)])
    key = autotune.batch_key(b)
    # an index past the current list, then a shape that no longer matches it
    for entry in ({"tile": 7, "shape": [32, 8]}, {"tile": 0, "shape": [32, 8]}):
        json.dump({key: entry}, open(cache, "w"))
        r = autotune.best_tile(b, cache_path=cache)
        assert r == {"tile": 1, "cached": False, "ms": [1.0] * len(SHAPES)}
        assert json.load(open(cache))[key] == {"tile": 1, "shape": [32, 8]}
    assert f.tuned == 2
