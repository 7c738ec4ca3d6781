"""Autotuner for the layout and launch shape of a set of games.

Every launch shape of the library (threads per CTA, CTAs per SM, unit buffer
bytes; ``cfr.shapes()``), both unit layouts (several levels per unit, or one
level per unit below a root unit) and both ways of launching a player's two
passes (one kernel or two) compute the same iteration.  Which one is
fastest depends on the games: their sizes, depths and how many share a batch.
``tune`` loads the games under each candidate, times a few CUDA-graph replays
of real iterations with CUDA events on the solver's stream, and returns the
fastest choice together with the whole table.  The games' state is discarded
afterwards; load the games again with the chosen ``shape`` / ``flat`` /
``passes``.

A choice can be kept in a JSON cache file keyed by the load's layout
signature (``signature``: the device, the variant, the graph length, the
number of games and the spread of their sizes, each rounded to a power of
two), so that a later load of the same kind of batch reuses it
without timing anything.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import cfr as C


def signature(trees, variant="cfr+", iterations=64) -> str:
    """Layout signature of a load: loads with equal signatures have the same
    number of games to within a factor of two and the same size histogram
    (games per power-of-two node count) to within a factor of two per
    bucket."""
    import torch

    ts = trees if isinstance(trees, (list, tuple)) else [trees]
    p2 = lambda v: int(math.floor(math.log2(max(1, v))))
    hist = {}
    for t in ts:
        b = p2(t.n_nodes)
        hist[b] = hist.get(b, 0) + 1
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    h = ",".join(f"{b}:{p2(n)}" for b, n in sorted(hist.items()))
    return f"{dev}|{variant}|k{iterations}|g{p2(len(ts))}|{h}"


def _cache_get(path, key):
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def _cache_put(path, key, entry):
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[key] = entry
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(trees, variant="cfr+", iterations=64, repeats=3, candidates=None, stream=None, budget_s=None,
         cache=None):
    """Time `repeats` x `iterations` iterations of `variant` on `trees` (one
    game or a list) for each (shape, flat, passes) candidate; returns
    {"shape", "flat", "passes", "us_per_iteration",
     "table": [(shape, flat, passes, us), ...], "signature", "cached"}.
    `budget_s` stops trying further candidates once that much wall time has
    been spent (the default shape is always tried first).  With `cache` (a
    JSON file path), a choice stored for the same signature is returned
    without timing, and a new choice is stored there."""
    import torch

    key = signature(trees, variant, iterations)
    if cache is not None:
        hit = _cache_get(cache, key)
        if hit is not None:
            return {**hit, "table": [tuple(r) for r in hit["table"]], "signature": key, "cached": True}
    if candidates is None:
        shapes = sorted(C.shapes())
        ts = trees if isinstance(trees, (list, tuple)) else [trees]
        default = C.pick_shape(len(ts), sum(t.n_nodes for t in ts))
        order = [default] + [k for k in shapes if k != default]
        candidates = [(k, flat, passes) for k in order for flat in (False, True) for passes in (1, 2)]
    st = stream if stream is not None else torch.cuda.Stream()
    t_start = time.perf_counter()
    table = []
    for shape, flat, passes in candidates:
        if budget_s is not None and table and time.perf_counter() - t_start > budget_s:
            break
        s = C.Solver(trees, stream=st, shape=shape, flat=flat, passes=passes)
        s.set_graph_iterations(iterations)
        s.iterate(iterations, variant)   # captures the graph, warms the caches
        s.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.iterate(repeats * iterations, variant)
        e1.record(st)
        e1.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / (repeats * iterations)
        s.close()
        table.append((shape, flat, passes, us))
    best = min(table, key=lambda r: r[3])
    out = {"shape": best[0], "flat": best[1], "passes": best[2], "us_per_iteration": best[3], "table": table}
    if cache is not None:
        _cache_put(cache, key, {**out, "table": [list(r) for r in table]})
    return {**out, "signature": key, "cached": False}
