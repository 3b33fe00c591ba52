"""Autotuning of the Fisher-pass tiles, with a JSON cache.

The fused point kernels take a tile: lanes per work item (4, 8 or 16) and CTAs
per SM of the persistent grid (1 or 2).  The best tile depends on the GPU, the
precision and the grid lengths of the catalog, so the library keeps one tile
per (precision, grid-length class) and ``gw_autotune`` times all six on a
catalog.  This module runs the tuner where the cache has no entry and stores
the winners in a JSON file keyed by device name and SM count, so that a later
process on the same kind of GPU installs them without timing anything.

Cache file: $GWFISH_AUTOTUNE_CACHE, else ~/.cache/gwfish/autotune.json.
"""
from __future__ import annotations

import json
import os

import torch

from . import (GW_FP64, GW_MIXED, LENGTH_CLASSES, gw_autotune, gw_set_tile, load_library,
               work_items)


def cache_path() -> str:
    return os.environ.get("GWFISH_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gwfish",
                                       "autotune.json"))


def device_key(device: int | None = None) -> str:
    """'<device name>|<SM count>|abi<library ABI version>'."""
    if device is None:
        device = torch.cuda.current_device()
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|{p.multi_processor_count}|abi{load_library().gw_abi_version()}"


def load(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _name(prec: int) -> str:
    return "mixed" if prec == GW_MIXED else "fp64"


def apply(cache: dict | None = None, device: int | None = None) -> int:
    """Install every cached tile of this device; returns how many."""
    cache = load() if cache is None else cache
    entries = cache.get(device_key(device), {})
    k = 0
    for prec in (GW_FP64, GW_MIXED):
        for cls, name in enumerate(LENGTH_CLASSES):
            t = entries.get(f"{_name(prec)}/{name}")
            if t:
                gw_set_tile(prec, cls, int(t["group"]), int(t["blocks_per_sm"]))
                k += 1
    return k


def length_class_of(npts) -> int:
    """Grid-length class of a catalog (the library's rule): mean work items of
    GW_ITEM_POINTS points per event, <= 1.5 -> 0, <= 12 -> 1, else 2."""
    n = int(torch.as_tensor(npts).numel())
    m = work_items(npts) / max(1, n)
    return 0 if m <= 1.5 else (1 if m <= 12.0 else 2)


def tune(cat, net, n_par: int, prec: int, reps: int = 3, path: str | None = None,
         force: bool = False) -> dict:
    """The tile of this catalog's grid-length class and precision: from the
    cache (installed without timing), or timed by gw_autotune and stored.
    Returns the entry (group, blocks_per_sm, ms per tile when timed, cached,
    length_class)."""
    npts = cat.npts if cat.sel is None else cat.npts[cat.sel]
    cls = length_class_of(npts)
    cache = load(path)
    key = device_key()
    name = f"{_name(prec)}/{LENGTH_CLASSES[cls]}"
    entry = cache.get(key, {}).get(name)
    if entry and not force:
        gw_set_tile(prec, cls, int(entry["group"]), int(entry["blocks_per_sm"]))
        return dict(entry, cached=True, length_class=cls)
    res = gw_autotune(cat, net, n_par, prec, reps)
    if res["length_class"] != cls:
        raise RuntimeError("grid-length class rule differs between the library and the cache")
    entry = {"group": res["group"], "blocks_per_sm": res["blocks_per_sm"],
             "ms": {f"{g}x{b}": v for (g, b), v in res["ms"].items()}}
    cache.setdefault(key, {})[name] = entry
    save(cache, path)
    return dict(entry, cached=False, length_class=cls)
