"""Persistent cache of the collide-stream launch shape chosen by the native
autotuners (``btdf_autotune``, ``btdf_batch_autotune``).

The timing itself runs in the library (CUDA events around whole steps on the
lattice's own state, which is restored afterwards).  This module only keys
the result by what decides it -- GPU, lattice shape, storage, layout, delta
function, marker count and library version -- and stores it in a JSON file,
so a later run on the same configuration applies the choice without timing.

Cache file: ``$BTDF_AUTOTUNE_CACHE`` if set, else
``~/.cache/btdf/autotune.json``.  Writes go through a temporary file and an
atomic rename.
"""
from __future__ import annotations

import json
import os
import tempfile
from typing import Callable, Dict, Optional

from . import btdf as B

CACHE_ENV = "BTDF_AUTOTUNE_CACHE"


def default_cache_path() -> str:
    p = os.environ.get(CACHE_ENV)
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "btdf", "autotune.json")


def device_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name()
    except Exception:
        pass
    return "unknown-gpu"


def lattice_key(lat, device: str) -> str:
    c = lat.cfg
    return (f"{device}|lattice|{c.nx}x{c.ny}|storage={c.storage}|layout={c.layout}|"
            f"delta={c.delta}|nf={c.nf}|markers={lat.marker_count}|lib={B.btdf_version()}")


def batch_key(bt, device: str) -> str:
    sizes = ",".join(f"{c.nx}x{c.ny}" for c in bt.cases)
    import hashlib
    h = hashlib.sha256(sizes.encode()).hexdigest()[:16]
    return (f"{device}|batch|n={len(bt.cases)}|sizes={h}|storage={bt.storage}|"
            f"lib={B.btdf_version()}")


class TuneCache:
    def __init__(self, path: Optional[str] = None):
        self.path = path or default_cache_path()
        self.entries: Dict[str, dict] = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    data = json.load(f)
                if isinstance(data, dict):
                    self.entries = data
            except (OSError, ValueError):
                self.entries = {}   # unreadable cache: start afresh

    def get(self, key: str) -> Optional[dict]:
        return self.entries.get(key)

    def put(self, key: str, value: dict) -> None:
        self.entries[key] = value
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".autotune.", suffix=".json")
        with os.fdopen(fd, "w") as f:
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def _tune(obj, key: str, cache: TuneCache, run: Callable[[], tuple], apply: Callable[[int], None],
          retune: bool) -> dict:
    hit = None if retune else cache.get(key)
    if hit is not None:
        apply(int(hit["variant"]))
        return dict(hit, cached=True)
    chosen, ms = run()   # the native autotuner leaves the chosen variant applied
    entry = {"variant": int(chosen), "ms_per_step": {str(k): v for k, v in ms.items()}}
    cache.put(key, entry)
    return dict(entry, cached=False)


def tune_lattice(lat, cache: Optional[TuneCache] = None, steps: int = 20, flush_l2: bool = True,
                 device: Optional[str] = None, retune: bool = False) -> dict:
    """Applies the cached launch shape for this lattice, timing it first on a
    cache miss.  Returns the cache entry with ``cached`` set."""
    cache = cache or TuneCache()
    key = lattice_key(lat, device or device_name())
    return _tune(lat, key, cache, lambda: lat.autotune(steps, flush_l2), lambda v: lat.tune(v, 0),
                 retune)


def tune_batch(bt, cache: Optional[TuneCache] = None, steps: int = 10, flush_l2: bool = False,
               device: Optional[str] = None, retune: bool = False) -> dict:
    """As tune_lattice for a ``Batch``."""
    cache = cache or TuneCache()
    key = batch_key(bt, device or device_name())
    return _tune(bt, key, cache, lambda: bt.autotune(steps, flush_l2), bt.tune, retune)
