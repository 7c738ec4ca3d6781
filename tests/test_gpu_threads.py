"""Contexts loaded and freed on worker threads while the main thread iterates.

A serving loop loads the next games on worker threads while it iterates the
live ones, and each new context captures its CUDA graph on its first
iterations.  The library runs its CUDA set-up work (the device part of a load,
graph capture and instantiation, freeing) under one process-wide lock, so a
load or free on another thread never invalidates a capture in progress.  Here
four threads load and free contexts without pause while the main thread
creates fresh contexts and iterates them through new graphs; every capture
must succeed and every context must compute what a context alone computes.
"""
import threading

import numpy as np
import pytest

from paper_2605_14277_b300 import games as G

pytestmark = pytest.mark.gpu


def test_loads_on_threads_while_capturing():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_14277_b300 import cfr as C

    trees = [G.sized_random_game(9000 + k, 20000) for k in range(5)]
    ref = C.Solver(trees[0])
    ref.set_graph_iterations(8)
    ref.iterate(32, "dcfr")
    want = ref.get_state(1)["r"]
    ref.close()

    n_threads = 4
    stop = threading.Event()
    ready = threading.Barrier(n_threads + 1)
    errors = []
    loads = [0] * n_threads

    def loader(k):
        try:
            # this thread's first CUDA calls happen before any capture below
            C.Solver(trees[1 + k]).close()
            ready.wait(timeout=120)
            while not stop.is_set():
                s = C.Solver(trees[1 + (loads[k] + k) % 4])
                s.sizes()
                s.close()
                loads[k] += 1
        except Exception as e:   # reported by the main thread
            errors.append(e)
            ready.abort()

    threads = [threading.Thread(target=loader, args=(k,)) for k in range(n_threads)]
    for t in threads:
        t.start()
    try:
        ready.wait(timeout=120)
        for _ in range(6):
            s = C.Solver(trees[0])
            s.set_graph_iterations(8)   # a fresh context: its graph is captured now
            s.iterate(32, "dcfr")
            got = s.get_state(1)["r"]
            s.close()
            assert np.array_equal(got, want)
    finally:
        stop.set()
        for t in threads:
            t.join()
    assert not errors, errors
    assert min(loads) > 0
