"""The serving loop with the real library: continuous batching on the GPU.

Requests of mixed sizes arrive in bursts while earlier ones are still
iterating; they share cohorts (batched contexts on their own streams),
rounds run without waiting on one another, and the unfinished games of
mostly-solved cohorts move, with their exact state, into the cohorts that
new arrivals form.  Each served request must end exactly as the same
request solved alone (rounds of 64 DCFR iterations until its FP64
exploitability is at most TARGET of its payoff range): the same iteration
count and the same exploitability, bit for bit.  A few served requests are
also handed to the FP64 oracle at their final state for one more iteration.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2605_14277_b300 import games as G
from paper_2605_14277_b300 import serving as S
from tests.parity_util import assert_elementwise, strategy_mismatch_ok

pytestmark = pytest.mark.gpu

TARGET = 1e-5   # exploitability target, relative to the payoff range


@pytest.fixture(scope="module")
def cfr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_14277_b300 import cfr as C
    return C


def requests():
    rng = np.random.default_rng(11)
    trees = [G.serving_request(900 + k, lo=1e3, hi=3e4) for k in range(30)]
    # bursts of six, each arriving while the previous ones iterate
    arrivals = np.repeat(np.arange(5) * 0.05, 6) + rng.uniform(0, 1e-3, 30)
    return S.make_requests(trees, arrivals)


def test_served_results_equal_alone_results(cfr):
    import torch
    finals = {}

    def on_complete(r, solver, k):
        finals[r.rid] = {p: solver.get_state(p, game=k) for p in (1, 2)}

    rq = requests()
    cfr.Solver(G.poker_game()).close()   # library loaded, device initialised
    # a tight target keeps games iterating for many rounds, finishing at
    # different times; repack_live near 1: a cohort with any solved game
    # moves its unfinished games into the next cohort that arrivals form
    pool = S.loader_pool(2, initializer=torch.cuda.set_device, initargs=(0,))
    try:
        srv = S.Server(lambda trees, st: cfr.Solver(trees, stream=st), hbm_budget=8e9, round_iters=64,
                       variant="dcfr", target_rel=TARGET, max_cohort=8, repack_live=0.999,
                       stream_factory=torch.cuda.Stream, on_complete=on_complete, loader=pool.submit)
        st = srv.run(rq, time_limit=300.0)
    finally:
        pool.shutdown()
    print(st)
    print([(r.rid, round(r.arrival, 4), round(r.admitted, 4), round(r.done, 4), r.iterations, r.moves) for r in rq])
    assert st["completed"] == len(rq) and st["rejected"] == 0
    assert st["moved_games"] > 0, "the bursts never made a cohort move its unfinished games"
    assert abs(srv.in_use) < 1.0
    print(f"served {st['completed']} requests in {st['cohorts']} cohorts, {st['moved_games']} moves")
    for r in rq:
        s = cfr.Solver(r.tree)
        it = 0
        while True:
            s.iterate(64, "dcfr")
            it += 64
            e = s.exploitability()[0]
            if e <= TARGET * r.payoff_range:
                break
        assert r.iterations == it, (r.rid, r.iterations, it, r.moves)
        assert r.exploitability == e, (r.rid, r.exploitability, e, r.moves)
        s.close()
    # the oracle at the final state of moved requests: one more iteration
    moved = [r for r in rq if r.moves > 0][:3]
    for r in moved:
        o = Oracle(r.tree)
        g = cfr.Solver(r.tree)
        for p in (1, 2):
            f = finals[r.rid][p]
            o.set_state(p, f["r"], f["b"], f["xbar"], f["t"])
            g.set_state(p, f["r"], f["b"], f["xbar"], f["t"])
        assert f["t"] == r.iterations
        o.iterate(1, "dcfr")
        g.iterate(1, "dcfr")
        for p in (1, 2):
            a, b = g.get_state(p), o.get_state(p)
            assert_elementwise(a["xbar"], b["xbar"], ("xbar", r.rid, p))
            _, na = o.infosets(p)
            assert strategy_mismatch_ok(a["b"], b["b"], b["r"], na) == 0
        g.close()


def test_copy_game_states_is_exact(cfr):
    """A game's state moved into another context (where it sits among other
    games) continues exactly as it would have in place."""
    trees = [G.serving_request(950 + k, lo=1e3, hi=2e4) for k in range(4)]
    a = cfr.Solver(trees)
    a.iterate(100, "dcfr")
    b = cfr.Solver([trees[2], G.poker_game(), trees[0]])
    b.copy_states_from(a, [0, 2], [2, 0])
    for s in (a, b):
        s.iterate(70, "dcfr")
    for ga, gb in ((2, 0), (0, 2)):
        for p in (1, 2):
            x, y = a.get_state(p, game=ga), b.get_state(p, game=gb)
            assert x["t"] == y["t"] == 170
            for k in ("r", "b", "xbar"):
                assert np.array_equal(x[k], y[k]), (ga, p, k)
    with pytest.raises(cfr.CFRError):
        b.copy_states_from(a, [1], [1])   # different games
