"""Autotuner cache for the stream-collide kernel variant.

The library's ``lb_autotune`` times every (nodes per thread, block size)
variant on a context's lattice and then the L2 prefetch distance of the
winner; this module remembers both per
(device, storage, channel dimensions) in a JSON file outside the repository
(``$LBIBM_CACHE`` or ``~/.cache/lbibm/autotune.json``) so later runs skip the
timing.
"""
from __future__ import annotations

import json
import os


def cache_path() -> str:
    return os.environ.get("LBIBM_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "lbibm", "autotune.json")


def _key(device: str, storage: str, dims) -> str:
    return f"{device}|{storage}|" + ";".join("x".join(str(v) for v in d) for d in dims)


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(sim, device: str, storage: str, repeats: int = 20, use_cache: bool = True):
    """Apply the cached variant for this lattice, or time all variants and cache the best."""
    key = _key(device, storage, sim.dims)
    table = _load() if use_cache else {}
    if key in table:
        npt, bs = table[key]["npt"], table[key]["bs"]
        try:
            sim.set_kernel_config(npt, bs)
            sim.set_prefetch(table[key].get("pf", 0))
            return {"npt": npt, "bs": bs, "pf": sim.prefetch(), "ms": table[key].get("ms"), "cached": True}
        except RuntimeError:
            pass   # a variant this library no longer offers: time them again
    npt, bs, ms = sim.autotune(repeats)
    pf = sim.prefetch()
    table = _load()
    table[key] = {"npt": npt, "bs": bs, "pf": pf, "ms": ms}
    try:
        os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
        tmp = cache_path() + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path())
    except OSError:
        pass
    return {"npt": npt, "bs": bs, "pf": pf, "ms": ms, "cached": False}
