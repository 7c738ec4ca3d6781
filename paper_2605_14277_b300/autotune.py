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
"""
from __future__ import annotations

import time

from . import cfr as C


def tune(trees, variant="cfr+", iterations=64, repeats=3, candidates=None, stream=None, budget_s=None):
    """Time `repeats` x `iterations` iterations of `variant` on `trees` (one
    game or a list) for each (shape, flat, passes) candidate; returns
    {"shape", "flat", "passes", "us_per_iteration",
     "table": [(shape, flat, passes, us), ...]}.
    `budget_s` stops trying further candidates once that much wall time has
    been spent (the default shape is always tried first)."""
    import torch

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
    return {"shape": best[0], "flat": best[1], "passes": best[2], "us_per_iteration": best[3], "table": table}
