"""Autotuned launch settings with a JSON cache keyed by GPU and workload class.

The tuning itself is native (rt_autotune: coordinate descent over the wave
capacity, the traversal loop parameters and the traversal block size, timed
with CUDA events on probe renders).  This module only keys, stores and
reloads the results: key = cache version | GPU name | triangles (rounded to 2
significant digits) | pixels (rounded likewise) | bands | depth.
"""
from __future__ import annotations

import json
import math
import os
from typing import Optional

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "spectral_rt", "autotune.json")


def _round2(x: int) -> int:
    if x <= 0:
        return 0
    e = int(math.floor(math.log10(x))) - 1
    return int(round(x / 10 ** e) * 10 ** e)


# Bumped whenever the tuned fields or their valid ranges change, so that
# entries written by an older library are not reused.
CACHE_VERSION = 2


def workload_key(gpu_name: str, n_tris: int, n_pixels: int, n_bands: int, depth: int) -> str:
    return f"v{CACHE_VERSION}|{gpu_name}|{_round2(n_tris)}|{_round2(n_pixels)}|{n_bands}|{depth}"


def load(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tuned_options(renderer, workload, probe_bands: int = 9, spp_probe: int = 1, cache_path: Optional[str] = DEFAULT_CACHE,
                  retune: bool = False):
    """Tuned render options for a workload: from the cache, else tuned on a
    probe (spp_probe samples of all views, probe_bands bands in the middle of
    the spectrum) and stored."""
    import torch
    name = torch.cuda.get_device_name(renderer.device)
    key = workload_key(name, workload.scene.n_tris, workload.n_pixels, workload.band_count, workload.depth)
    cache = load(cache_path) if cache_path else {}
    if not retune and key in cache:
        return cache[key]["opts"], cache[key]
    nb = min(probe_bands, workload.band_count)
    first = workload.band_first + (workload.band_count - nb) // 2
    opts, report = renderer.autotune(workload.cameras, workload.depth, band_first=first, band_count=nb,
                                     spp_probe=spp_probe)
    entry = {"opts": opts, "report": report, "probe": {"bands": nb, "spp": spp_probe}}
    if cache_path:
        cache[key] = entry
        save(cache, cache_path)
    return opts, entry
