"""Autotuned launch shape of a batch, cached on disk.

The measurement is the library's own amlbm_autotune (every compiled schedule and
tile of the storage form, timed with CUDA events on the batch's lattice shapes).
Its choice is kept in a JSON file keyed by the GPU, the library version, the
storage form and the instances' shapes and flags, so that a later batch of the
same shapes starts without re-timing.  The file is $AMLBM_TUNE_CACHE, else
~/.cache/amlbm/autotune.json; AMLBM_TUNE_CACHE=off disables the cache.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

from . import amlbm

_lock = threading.Lock()


def cache_path():
    p = os.environ.get("AMLBM_TUNE_CACHE")
    if p == "off":
        return None
    return p or os.path.join(os.path.expanduser("~"), ".cache", "amlbm", "autotune.json")


def signature(specs, storage, device_name, version):
    """Key of a tuning: what the step's speed depends on (not tau, G or the fields)."""
    shapes = [[int(s.Nz), int(s.Nr), bool(s.axisym), str(s.src), str(s.wall), str(s.shift),
               str(s.rounding), float(s.gz) != 0.0, str(s.forcing), str(s.z_bc), str(s.r_lo)] for s in specs]
    blob = json.dumps({"device": device_name, "version": version, "storage": storage, "shapes": shapes},
                      sort_keys=True)
    return hashlib.sha256(blob.encode()).hexdigest()[:32]


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, key, entry):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    data = _load(path)
    data[key] = entry
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(specs, storage, steps=20, stream=None, use_cache=True):
    """{"schedule", "tile", "candidates", "cached"} for these lattices."""
    import torch
    lib = amlbm.load()
    dev = torch.cuda.get_device_name()
    key = signature(specs, storage, dev, lib.amlbm_version().decode())
    path = cache_path() if use_cache else None
    with _lock:
        if path:
            hit = _load(path).get(key)
            if hit:
                return dict(hit, cached=True)
        sched, tile, cands = amlbm.autotune_raw(specs, storage, steps=steps, stream=stream)
        entry = {"schedule": sched, "tile": list(tile), "candidates": cands, "storage": storage,
                 "device": dev, "steps": steps}
        if path:
            try:
                _store(path, key, entry)
            except OSError:
                pass  # a read-only home directory only costs the re-timing
        return dict(entry, cached=False)
