"""Tile-shape choice with a cache on disk.

``best_tile(batch)`` runs the library's autotuner (``lbm_autotune``: every
step-kernel shape timed on the batch's own lattices, state saved and
restored) the first time a kind of batch is seen, and keeps the winner in a
JSON file keyed by the GPU's name, the storage precision and the batch's
signature (each lattice's size, walls and pseudopotential kind). Later calls
for the same key select the cached shape without timing anything.
"""
import json
import os
from typing import Optional

from . import lbm

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pplbm_tiles.json")


def batch_key(batch: "lbm.Batch") -> str:
    import torch
    gpu = torch.cuda.get_device_name(torch.cuda.current_device())
    lats = sorted((s.nx, s.ny, s.solid is not None, getattr(s, "eos", "cs")) for s in batch.specs)
    return json.dumps({"gpu": gpu, "precision": int(batch.precision), "lattices": lats}, sort_keys=True)


def best_tile(batch: "lbm.Batch", steps: int = 20, cache_path: Optional[str] = None) -> dict:
    """Select the fastest tile shape for `batch`; returns {"tile": index,
    "cached": bool, "ms": per-shape times when measured}."""
    path = cache_path or DEFAULT_CACHE
    key = batch_key(batch)
    cache = {}
    if os.path.exists(path):
        with open(path) as fh:
            cache = json.load(fh)
    entry = cache.get(key)
    if entry is not None and 0 <= entry["tile"] < lbm.lbm_tile_count() and \
            list(lbm.lbm_tile_shape(entry["tile"])) == entry["shape"]:
        lbm.lbm_set_tile(batch.ctx, entry["tile"])
        return {"tile": entry["tile"], "cached": True, "ms": None}
    tile, ms = lbm.lbm_autotune(batch.ctx, steps)
    cache[key] = {"tile": tile, "shape": list(lbm.lbm_tile_shape(tile))}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1)
    os.replace(tmp, path)
    return {"tile": tile, "cached": False, "ms": ms}
