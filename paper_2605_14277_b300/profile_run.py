"""Run a few eager CFR iterations of a seeded workload, for external profilers.

    python -m paper_2605_14277_b300.profile_run --workload large --iters 3

Every iteration is launched directly (no CUDA graph), so a profiler sees the
four kernels of each iteration as separate launches in order:
player-1 up, player-1 down, player-2 up, player-2 down.
"""
from __future__ import annotations

import argparse

from . import games as G


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="large", choices=["large", "poker", "batch"])
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--variant", default="dcfr")
    ap.add_argument("--batch-games", type=int, default=256)
    args = ap.parse_args()
    import torch
    from . import cfr as C
    torch.cuda.set_device(0)
    if args.workload == "large":
        trees = G.large_random_game(3)
    elif args.workload == "poker":
        trees = G.poker_game()
    else:
        trees = G.batch_games(args.batch_games)
    s = C.Solver(trees)
    s.set_graph_iterations(4096)
    s.iterate(args.iters, args.variant)
    s.sync()
    print("done", args.workload, args.iters, s.sizes())


if __name__ == "__main__":
    main()
