"""Persistent cache of the contraction autotuner's picks (p2s_autotune_tiles).

A tile configuration depends on the batch's shape, not on its values: the multiset of
per-element orders, the quadrature rule, the precision, the product types and the GPU.
The cache keys a pick by that signature and stores it as JSON, so a batch of a shape
already tuned on a device of the same name skips the tuning.  Two files are consulted:

  - the shipped table next to this module (``tiles.json``), with picks measured on the
    devices this library was tuned on;
  - a user table, ``$P2S_TUNE_CACHE`` or ``~/.cache/p2s/tiles.json``, where new picks are
    written.

The cache holds host logic only (no arithmetic of the method).
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

import numpy as np

SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiles.json")


def user_path() -> str:
    return os.environ.get("P2S_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "p2s", "tiles.json")


def signature(orders, npts, precision, types_mask, device_name) -> str:
    """Key of a batch shape: device, precision, types, the histogram of quadrature sizes and
    a digest of the histogram of per-element order tuples (element order does not matter)."""
    o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(np.asarray(orders).shape[0], -1))
    E = o.shape[0]
    g = np.broadcast_to(np.asarray(npts, dtype=np.int64), (E,))
    rows, counts = np.unique(o, axis=0, return_counts=True) if E else (o, np.zeros(0, np.int64))
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(rows, dtype=np.int32).tobytes())
    h.update(np.ascontiguousarray(counts, dtype=np.int64).tobytes())
    gv, gc = np.unique(g, return_counts=True) if E else (g, np.zeros(0, np.int64))
    ghist = ",".join("%d:%d" % (int(a), int(b)) for a, b in zip(gv, gc))
    return "%s|p%d|t%d|E%d|G%s|o%s" % (device_name, int(precision), int(types_mask), E, ghist, h.hexdigest()[:16])


def _read(path):
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def lookup(key):
    """The cached entry for `key` ({"tile": {...}, ...}), user table first, or None."""
    for path in (user_path(), SHIPPED):
        e = _read(path).get(key)
        if e and isinstance(e.get("tile"), dict):
            return e
    return None


def store(key, entry, path=None):
    """Add `entry` under `key` to the user table (atomic replace of the file)."""
    path = path or user_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    d = _read(path)
    d[key] = entry
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path), suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned_tile(tune, key, **meta):
    """The tile for `key`: from the cache, else `tune()` -> (tile, best_ms, tried) and stored.
    Returns (tile, info) with info["cache"] = "hit" or "miss"."""
    e = lookup(key)
    if e is not None:
        return e["tile"], dict(e, cache="hit", key=key)
    tile, best_ms, tried = tune()
    entry = dict(meta, tile=tile, sample_contract_ms=best_ms, candidates=tried)
    try:
        store(key, entry)
    except OSError:
        pass
    return tile, dict(entry, cache="miss", key=key)
