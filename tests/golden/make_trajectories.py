"""Write the trajectory fixtures tests/golden/trajectory_*.json.

Every stored value comes from the FP64 CPU oracle (oracle/) alone, run on the
seeded synthetic games of paper_2605_14277_b300/games.py; nothing here calls
the CUDA library.  For each workload the oracle runs the stated variant from
the initial state (r = 0, uniform strategies) and records the exploitability
(BR1 + BR2) / 2 of the average strategies (Sec. 4's metric; the paper gives no
formula, this is the reading the oracle implements) at each checkpoint.  The
same run is repeated on reordered copies of each game (tests/parity_util.py
`reorder`: nodes renumbered, infoset ids permuted), which change only the
order of the oracle's FP64 summations; the spread of those runs is the
oracle's own sensitivity to rounding along a trajectory (Appendix D).

    python tests/golden/make_trajectories.py [names...]    # default: all

Names: small_cfr, poker, batch_cfrplus, large_dcfr (the last takes about 15
minutes per run on one core; its runs go to separate processes).
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.oracle import Oracle  # noqa: E402
from paper_2605_14277_b300 import games as G  # noqa: E402
from tests.parity_util import reorder  # noqa: E402

N_REORDER = {"small_cfr": 8, "poker": 96, "batch_cfrplus": 12, "large_dcfr": 2}
# batch games whose first runs spread wider than 1e-3 get this many reorderings
N_REORDER_WIDE = 96


def trajectory(tree, variant, checkpoints, reorder_seed=None, params=None):
    """Exploitability of the oracle's averages at each checkpoint."""
    t = tree if reorder_seed is None else reorder(tree, reorder_seed)
    o = Oracle(t)
    out, done = [], 0
    for c in checkpoints:
        o.iterate(c - done, variant, **(params or {}))
        done = c
        out.append(o.exploitability()[0])
    return out


def _large_run(seed):
    return trajectory(G.large_random_game(3), "dcfr", [1000, 5000, 10000], seed)


def runs_of(make_tree, variant, checkpoints, n_reorder):
    runs = {"base": trajectory(make_tree(), variant, checkpoints)}
    for k in range(1, n_reorder + 1):
        runs[f"reorder{k}"] = trajectory(make_tree(), variant, checkpoints, k)
    return runs


def make_small():
    cps = list(range(100, 1001, 100))
    return {"workload": "small_random_d6_s1 (games.small_random_game(1))", "variant": "cfr",
            "params": "alpha 0, beta 0, gamma 0 (uniform average), simultaneous updates",
            "checkpoints": cps, "runs": runs_of(lambda: G.small_random_game(1), "cfr", cps, N_REORDER["small_cfr"])}


def make_poker():
    cps = [1000, 5000, 10000]
    out = {"workload": "poker_6card_2round (games.poker_game())", "checkpoints": cps, "variants": {}}
    for v in ("cfr+", "dcfr", "pcfr+", "pcfr"):
        out["variants"][v] = runs_of(G.poker_game, v, cps, N_REORDER["poker"])
    out["params"] = "library defaults: cfr+ (gamma 1), dcfr (1.5, 0, 2), pcfr+ (gamma 2), pcfr (gamma 0); alternating"
    return out


def make_batch():
    seeds = G.batch_sample_seeds(64)
    cps = [1024]
    games = {}
    for s in seeds:
        runs = runs_of(lambda s=s: G.batch_game(s), "cfr+", cps, N_REORDER["batch_cfrplus"])
        vals = [r[-1] for r in runs.values()]
        if max(vals) / min(vals) - 1.0 > 1e-3:
            # a game whose trajectory depends on rounding: sample the spread wider
            for k in range(N_REORDER["batch_cfrplus"] + 1, N_REORDER_WIDE + 1):
                runs[f"reorder{k}"] = trajectory(G.batch_game(s), "cfr+", cps, k)
        games[str(s)] = runs
    return {"workload": "64-game sample of the 4096-game batch (games.batch_game(seed), seeds batch_sample_seeds(64))",
            "variant": "cfr+", "params": "gamma 1, alternating", "checkpoints": cps, "games": games}


def make_large():
    seeds = [None] + list(range(1, N_REORDER["large_dcfr"] + 1))
    with mp.get_context("spawn").Pool(len(seeds)) as pool:
        res = pool.map(_large_run, seeds)
    runs = {"base": res[0]}
    for k, r in enumerate(res[1:], 1):
        runs[f"reorder{k}"] = r
    return {"workload": "large_random_d12_s3 (games.large_random_game(3))", "variant": "dcfr",
            "params": "alpha 1.5, beta 0, gamma 2, alternating", "checkpoints": [1000, 5000, 10000], "runs": runs}


MAKERS = {"small_cfr": make_small, "poker": make_poker, "batch_cfrplus": make_batch, "large_dcfr": make_large}


def main(names):
    for name in names or list(MAKERS):
        t0 = time.time()
        d = MAKERS[name]()
        d["source"] = ("FP64 CPU oracle (oracle/cfr_oracle.c) from the initial state; exploitability = "
                       "(BR1 + BR2) / 2 of the normalised averages; reorderN = the same game with nodes and "
                       "infosets renumbered by tests/parity_util.reorder(tree, N) (summation order only); "
                       "written by tests/golden/make_trajectories.py")
        path = os.path.join(HERE, f"trajectory_{name}.json")
        with open(path, "w") as f:
            json.dump(d, f, indent=1)
        print(f"{name}: {time.time() - t0:.1f} s -> {path}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
