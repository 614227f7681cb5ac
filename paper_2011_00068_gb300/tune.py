"""Launch-shape autotuner for the walk.

The walk's results do not depend on its launch shape (walkers per CTA, steps per
chunk launch): the parity tests check that every shape gives bit-identical
trajectories.  Speed does depend on it, through occupancy, the tail of each chunk
launch and launch overhead, so this module times short walks of the actual walker mix
for each candidate shape on the current GPU and keeps the fastest.  Results are cached
in a JSON file next to the built library, keyed by GPU name, lengths and walker counts.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import build as _build

CACHE = os.path.join(_build.OUT_DIR, "tune_cache.json")
WARPS = (2, 4, 8)
CHUNKS = (256, 1024, 4096)
_lock = threading.Lock()


def _key(Ls, walkers, tabu_log2, dev) -> str:
    name = torch.cuda.get_device_name(dev)
    return "%s|%s|%s|%d" % (name, ",".join(map(str, Ls)), ",".join(map(str, walkers)), tabu_log2)


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(Ls, walkers, *, seed: int = 0, tabu_log2: int = 16, steps: int = 512, device=None,
         refresh: bool = False, flags: int = 0) -> dict:
    """Fastest {"warps_per_cta", "chunk_steps"} for this length mix on this GPU (flags:
    the context flags that change the kernel, e.g. LABS_FLAG_BEST_FIRST)."""
    from . import Search

    Ls = list(Ls) if isinstance(Ls, (list, tuple)) else [int(Ls)]
    walkers = list(walkers) if isinstance(walkers, (list, tuple)) else [int(walkers)]
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    key = _key(Ls, walkers, tabu_log2, dev) + ("" if not flags else "/flags%d" % flags)
    with _lock:
        cache = _load()
        if key in cache and not refresh:
            return cache[key]
    timings = {}
    multi = len(Ls) > 1
    for wpc in WARPS:
        for chunk in CHUNKS:
            # the shape is fixed at context creation: one context per candidate
            s = Search(Ls if multi else Ls[0], walkers if multi else walkers[0], seed, device=dev,
                       tabu_log2=tabu_log2, warps_per_cta=wpc, chunk_steps=chunk, flags=flags)
            s.walk(min(steps, 64))  # warm-up: graph capture, first touch of the tables
            s.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s.stream)
            s.walk(steps)
            b.record(s.stream)
            s.sync()
            timings[(wpc, chunk)] = a.elapsed_time(b)
            s.close()
    (wpc, chunk), ms = min(timings.items(), key=lambda kv: kv[1])
    best = {"warps_per_cta": wpc, "chunk_steps": chunk, "ms": ms,
            "all": {"%d/%d" % k: v for k, v in sorted(timings.items())}}
    with _lock:
        cache = _load()
        cache[key] = best
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + ".%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, CACHE)
    return best
