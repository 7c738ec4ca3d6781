"""Serving loop host logic (admission under a budget, rounds, completion at
the exploitability target, cohort release) with a stand-in solver: CPU only."""
import numpy as np

from paper_2605_14277_b300 import games as G
from paper_2605_14277_b300 import serving as S


class FakeClock:
    def __init__(self, dt=1e-4):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeRound:
    """A round whose result is ready after a few polls."""

    def __init__(self, e, polls=2):
        self.e, self.left = e, polls

    def done(self):
        self.left -= 1
        return self.left < 0

    def result(self):
        return self.e


class FakeSolver:
    """exploitability of game k after n iterations: range_k * c_k / n, with
    c_k = 0.5 unless `spread` varies it by game; a 1e-3 target is then met
    after 512 iterations; holds 100 bytes per node."""
    log = []
    spread = False

    def __init__(self, trees, stream=None):
        self.trees = trees
        self.n = np.zeros(len(trees))
        self.ranges = np.array([S.payoff_range(t) for t in trees])
        self.c = np.array([0.05 + 0.2 * (t.n_nodes % 7) if FakeSolver.spread else 0.5 for t in trees])
        self.closed = False
        FakeSolver.log.append(self)
        self.masks = []

    def iterate(self, n, variant="dcfr", active=None):
        a = np.ones(len(self.trees), bool) if active is None else np.asarray(active, bool)
        self.masks.append(a.copy())
        self.n[a] += n

    def exploitability_batch(self):
        e = self.ranges * self.c / np.maximum(self.n, 1)
        return e, e, e

    def start_round(self, n, variant="dcfr", active=None):
        assert not self.closed
        self.iterate(n, variant, active)
        return FakeRound(self.exploitability_batch()[0].copy())

    def copy_states_from(self, src, dst_games, src_games):
        assert not src.closed and not self.closed
        for d, k in zip(dst_games, src_games):
            assert src.trees[k] is self.trees[d]
            self.n[d] = src.n[k]

    def sizes(self, g=0):
        return {"device_bytes": 100 * sum(t.n_nodes for t in self.trees)}

    def close(self):
        self.closed = True


def reqs(n=12, rate=2000.0):
    trees = [G.small_random_game(s) for s in range(n)]
    return S.make_requests(trees, G.poisson_arrivals(5, rate, n))


def test_all_requests_complete_at_their_target():
    FakeSolver.log = []
    rq = reqs()
    srv = S.Server(FakeSolver, hbm_budget=1e12, round_iters=64, clock=FakeClock())
    st = srv.run(rq)
    assert st["completed"] == len(rq)
    for r in rq:
        assert r.done >= r.admitted >= r.arrival
        assert r.iterations == 512          # first multiple of 64 with 0.5/n <= 1e-3
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    assert st["solves_per_s"] > 0
    assert all(s.closed for s in FakeSolver.log)
    assert abs(srv.in_use) < 1.0


def test_budget_limits_what_is_resident():
    FakeSolver.log = []
    rq = reqs(8)
    one = max(r.nodes for r in rq) * 100
    srv = S.Server(FakeSolver, hbm_budget=1.5 * one, round_iters=64, bytes_per_node=100.0, clock=FakeClock())
    st = srv.run(rq)
    assert st["completed"] == len(rq)
    assert st["peak_bytes"] <= 1.5 * one
    assert st["cohorts"] >= 2 and st["rejected"] == 0


def test_request_larger_than_the_budget_is_rejected():
    FakeSolver.log = []
    rq = reqs(4)
    big = max(rq, key=lambda r: r.nodes)
    srv = S.Server(FakeSolver, hbm_budget=big.nodes * 100 - 1, bytes_per_node=100.0, clock=FakeClock())
    st = srv.run(rq)
    assert st["rejected"] >= 1 and big.done < 0
    assert st["completed"] == len(rq) - st["rejected"]


def test_no_request_is_admitted_before_it_arrives_and_done_games_are_masked():
    FakeSolver.log = []
    rq = reqs(6, rate=50.0)          # arrivals spread out
    srv = S.Server(FakeSolver, hbm_budget=1e12, round_iters=64, clock=FakeClock(1e-3))
    srv.run(rq)
    for r in rq:
        assert r.admitted >= r.arrival
    # a cohort of several games: once a game is done its slot is masked off
    for s in FakeSolver.log:
        seen_done = np.zeros(len(s.trees), bool)
        for m in s.masks:
            assert not (m & seen_done).any()
            seen_done |= ~m


def test_mixed_sizes_finish_in_a_shared_cohort():
    FakeSolver.log = []
    trees = [G.small_random_game(1), G.poker_game(), G.rps()]
    rq = S.make_requests(trees, [0.0, 0.0, 0.0])
    srv = S.Server(FakeSolver, hbm_budget=1e12, clock=FakeClock())
    st = srv.run(rq)
    assert st["completed"] == 3 and st["cohorts"] == 1


def alone_iterations(r, c_of):
    c = c_of(r.tree)
    need = c / 1e-3                     # range * c / n <= 1e-3 * range
    return int(np.ceil(need / 64.0) * 64)


def test_unfinished_games_move_to_new_cohorts_and_memory_returns():
    """Games of one cohort finish at different times; once most of a cohort
    is solved, its unfinished games move into the next cohort formed from new
    arrivals, with their state, and the old cohort's memory is returned.
    Every request still takes exactly the iterations it takes alone."""
    FakeSolver.log = []
    FakeSolver.spread = True
    try:
        trees = [G.sized_random_game(7000 + k, 200 + 37 * k) for k in range(40)]
        rq = S.make_requests(trees, np.repeat(np.arange(5) * 0.008, 8))   # five bursts of eight
        srv = S.Server(FakeSolver, hbm_budget=1e12, round_iters=64, max_cohort=8, clock=FakeClock(2e-4),
                       repack_live=0.6)
        st = srv.run(rq)
        assert st["completed"] == len(rq)
        assert st["moved_games"] > 0
        assert all(s.closed for s in FakeSolver.log) and srv.in_use == 0
        c_of = lambda t: 0.05 + 0.2 * (t.n_nodes % 7)
        for r in rq:
            assert r.iterations == alone_iterations(r, c_of), (r.rid, r.iterations, r.moves)
        assert any(r.moves > 0 for r in rq)
    finally:
        FakeSolver.spread = False


def test_one_at_a_time_baseline():
    rq = reqs(5)
    st = S.serve_one_at_a_time(FakeSolver, rq, clock=FakeClock())
    assert st["completed"] == 5
    assert all(r.iterations == 512 for r in rq)


def test_background_loader():
    from concurrent.futures import ThreadPoolExecutor
    FakeSolver.log = []
    rq = reqs(10)
    with ThreadPoolExecutor(max_workers=2) as pool:
        srv = S.Server(FakeSolver, hbm_budget=1e12, max_cohort_nodes=1500, clock=FakeClock(),
                       loader=pool.submit)
        st = srv.run(rq)
    assert st["completed"] == len(rq)
    assert st["cohorts"] >= 2          # the node cap splits the arrivals
    assert abs(srv.in_use) < 1.0


def test_loader_pool_starts_every_thread_first():
    # every pool thread exists and has run its initializer before the pool is
    # handed to the server (a late-starting thread's first CUDA calls could
    # invalidate a graph capture in progress)
    import threading
    seen = []
    lock = threading.Lock()

    def init(tag):
        with lock:
            seen.append((tag, threading.get_ident()))

    pool = S.loader_pool(5, initializer=init, initargs=("dev0",))
    try:
        assert len(seen) == 5 and len({t for _, t in seen}) == 5 and all(tag == "dev0" for tag, _ in seen)
        # later work reuses those threads
        ids = set(pool.map(lambda _: threading.get_ident(), range(20)))
        assert ids <= {t for _, t in seen}
    finally:
        pool.shutdown()
