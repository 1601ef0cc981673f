"""Autotuner of the phase kernels' grid sizes (blocks per SM per kernel kind).

The four phase kernels (primitives, gradients, fluxes, updates) grid-stride
over level-sorted ranges whose sizes vary by phase and by workload, so the
best number of resident blocks is workload dependent.  Results do not depend
on the choice (every item is computed independently), so the tuner simply
times candidates: coordinate descent over the kinds, a few candidate values
each, each candidate timed over whole cycles with CUDA events on the
caller's stream.  The choice is cached in a JSON file keyed by GPU name and
workload signature.

Each timed candidate advances the mesh (or batch) by a few cycles; pass
`reset` (a callable that sets the state again) to start every candidate from
the same state, which also keeps strong flows from being run past their valid
time while tuning.
"""
from __future__ import annotations

import json
import os

KINDS = ("prim", "grad", "flux", "update")
CANDIDATES = {"prim": (4, 8, 16), "grad": (4, 8, 16), "flux": (8, 16, 32), "update": (4, 8, 16)}
ORDER = (2, 3, 1, 0)  # flux, update, grad, prim: largest shares first

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_cycles(torch, target, stream, reps, reset=None):
    if reset is not None:
        reset()
    target.advance(1, stream=stream) if hasattr(target, "meshes") else \
        target.advance(1, stream=stream, want_time=False)          # capture + warm
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        if hasattr(target, "meshes"):
            target.advance(1, stream=stream)
        else:
            target.advance(1, stream=stream, want_time=False)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def autotune(target, signature: str, stream=None, reps: int = 3, cache_path: str = CACHE,
             use_cache: bool = True, reset=None):
    """Pick and apply blocks-per-SM for a fv.Mesh or fv.Batch.

    Returns (per_sm list, {"ms": best ms per cycle or None if cached,
    "tried": [(per_sm, ms), ...], "cached": bool})."""
    import torch
    gpu = torch.cuda.get_device_name(torch.cuda.current_device())
    key = f"{gpu}|{signature}"
    cache = _load(cache_path) if use_cache else {}
    if use_cache and key in cache:
        best = [int(x) for x in cache[key]["per_sm"]]
        target.set_launch(best)
        return best, {"ms": cache[key].get("ms"), "tried": [], "cached": True}
    if stream is None:
        stream = torch.cuda.Stream()
    best = list(target.get_launch())
    target.set_launch(best)
    best_ms = _time_cycles(torch, target, stream, reps, reset)
    tried = [(list(best), best_ms)]
    for k in ORDER:
        for v in CANDIDATES[KINDS[k]]:
            cand = list(best)
            cand[k] = v
            if any(cand == t for t, _ in tried):  # timed already
                continue
            target.set_launch(cand)
            ms = _time_cycles(torch, target, stream, reps, reset)
            tried.append((cand, ms))
            if ms < best_ms:
                best, best_ms = cand, ms
    target.set_launch(best)
    cache = _load(cache_path)
    cache[key] = {"per_sm": best, "ms": best_ms}
    _store(cache_path, cache)
    return best, {"ms": best_ms, "tried": tried, "cached": False}
