"""Serving loop: subgame-solve requests admitted under an HBM budget and
iterated until each meets its exploitability target.

Requests arrive over time (each a game tree).  The loop:

* admits the requests that have arrived, as one *cohort* (one batched
  context on its own CUDA stream), while the cohort's estimated device bytes
  fit the remaining budget;
* advances every live cohort by a round of K iterations, with the games that
  are already solved masked off;
* after each round reads the FP64 exploitability of every game of the cohort
  and completes the games at or below ``target_rel`` x (max payoff - min
  payoff), recording completion time - arrival time as the request's latency;
* frees a cohort once all its games are done, returning its bytes to the
  budget.

Every CFR step runs in the library (through ``cfr.Solver``); this module is
host-side scheduling only.  ``solver_factory`` lets the tests drive the loop
with a stand-in that needs no GPU.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float        # seconds after the start of the run
    tree: object          # games.Tree
    nodes: int
    payoff_range: float
    admitted: float = -1.0
    done: float = -1.0
    iterations: int = 0

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def payoff_range(tree) -> float:
    term = tree.kind == 3
    if not term.any():
        return 0.0
    p = tree.payoff[term]
    return float(p.max() - p.min())


def make_requests(trees, arrivals) -> List[Request]:
    return [Request(k, float(a), t, int(t.n_nodes), payoff_range(t)) for k, (t, a) in enumerate(zip(trees, arrivals))]


class Cohort:
    def __init__(self, reqs: List[Request], solver, est_bytes: int):
        self.reqs = reqs
        self.solver = solver
        self.active = np.ones(len(reqs), dtype=np.uint8)
        self.bytes = est_bytes
        self.iterations = 0

    @property
    def finished(self) -> bool:
        return not self.active.any()


class Server:
    """`solver_factory(trees, stream)` returns an object with the Solver
    methods iterate(n, variant, active=mask), exploitability_batch(), sizes()
    and close().  `stream_factory()` returns a stream per cohort (or None)."""

    def __init__(self, solver_factory: Callable, hbm_budget: float = 120e9, round_iters: int = 64,
                 variant: str = "dcfr", target_rel: float = 1e-3, bytes_per_node: float = 90.0,
                 max_cohort: int = 4096, max_cohort_nodes: float = 4e6, stream_factory: Optional[Callable] = None,
                 clock: Callable[[], float] = time.perf_counter, max_iterations: int = 100000,
                 loader: Optional[Callable] = None):
        self.factory = solver_factory
        self.budget = float(hbm_budget)
        self.round_iters = int(round_iters)
        self.variant = variant
        self.target_rel = float(target_rel)
        self.bytes_per_node = float(bytes_per_node)
        self.max_cohort = int(max_cohort)
        self.max_cohort_nodes = float(max_cohort_nodes)
        self.stream_factory = stream_factory or (lambda: None)
        # loader(fn) -> a future-like object with done() and result(); None
        # loads synchronously in the scheduling loop.  A thread pool's threads
        # should all exist, with their device set up, before run() (see
        # loader_pool): a thread's first CUDA calls can invalidate a CUDA-graph
        # capture that the scheduling loop has in progress
        self.loader = loader
        self.clock = clock
        self.max_iterations = int(max_iterations)
        self.cohorts: List[Cohort] = []
        self.in_use = 0.0
        self.peak_in_use = 0.0
        self.n_cohorts = 0
        self.rejected: List[Request] = []

    def _wait_until(self, t0: float, t: float):
        while True:
            left = t - (self.clock() - t0)
            if left <= 0:
                return
            if self.clock is time.perf_counter:
                time.sleep(min(left, 1e-3))

    def estimate(self, req: Request) -> float:
        return req.nodes * self.bytes_per_node

    def _admit(self, pending: List[Request], now: float) -> List[Request]:
        """Take arrived requests, in arrival order, while they fit the budget.
        A request larger than the whole budget can never be admitted: it is
        rejected (done stays negative, counted in the stats)."""
        take = []
        room = self.budget - self.in_use
        nodes = 0
        while pending and pending[0].arrival <= now and len(take) < self.max_cohort:
            need = self.estimate(pending[0])
            if need > self.budget:
                self.rejected.append(pending.pop(0))
                continue
            if need > room or (take and nodes + pending[0].nodes > self.max_cohort_nodes):
                break
            room -= need
            nodes += pending[0].nodes
            take.append(pending.pop(0))
        return take

    def _complete(self, c: Cohort, expl: np.ndarray, now: float):
        for k, r in enumerate(c.reqs):
            if not c.active[k]:
                continue
            r.iterations = c.iterations
            if expl[k] <= self.target_rel * r.payoff_range or c.iterations >= self.max_iterations:
                c.active[k] = 0
                r.done = now

    def _start(self, c: Cohort, t0: float):
        """A loaded cohort joins the rounds; its bytes are re-counted from what
        the library really holds."""
        real = float(c.solver.sizes()["device_bytes"])
        self.bytes_per_node = max(self.bytes_per_node, real / max(1, sum(r.nodes for r in c.reqs)))
        self.in_use += max(real, c.bytes) - c.bytes
        c.bytes = max(real, c.bytes)
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        now = self.clock() - t0
        for r in c.reqs:
            r.admitted = now
        self.cohorts.append(c)

    def run(self, requests: List[Request], time_limit: float = float("inf")) -> dict:
        pending = sorted(requests, key=lambda r: r.arrival)
        loading = []   # (future, cohort without solver)
        t0 = self.clock()
        while pending or self.cohorts or loading:
            now = self.clock() - t0
            if now > time_limit:
                break
            # admit what has arrived, as cohorts under the budget (bytes are
            # counted from admission on)
            while True:
                take = self._admit(pending, now)
                if not take:
                    break
                c = Cohort(take, None, sum(self.estimate(r) for r in take))
                self.in_use += c.bytes
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                self.n_cohorts += 1
                trees, stream = [r.tree for r in take], self.stream_factory()
                if self.loader is None:
                    c.solver = self.factory(trees, stream)
                    self._start(c, t0)
                else:
                    loading.append((self.loader(lambda ts=trees, st=stream: self.factory(ts, st)), c))
            for item in [x for x in loading if x[0].done()]:
                loading.remove(item)
                item[1].solver = item[0].result()
                self._start(item[1], t0)
            if not self.cohorts:
                if loading:
                    time.sleep(2e-4) if self.clock is time.perf_counter else None
                elif pending:   # nothing resident: wait for the next arrival
                    self._wait_until(t0, pending[0].arrival)
                continue
            # one round for every live cohort (asynchronous on their streams),
            # then the exploitability of each cohort's games
            for c in self.cohorts:
                c.solver.iterate(self.round_iters, self.variant, active=c.active)
                c.iterations += self.round_iters
            for c in self.cohorts:
                expl, _, _ = c.solver.exploitability_batch()
                self._complete(c, expl, self.clock() - t0)
            for c in [c for c in self.cohorts if c.finished]:
                c.solver.close()
                self.in_use -= c.bytes
                self.cohorts.remove(c)
        return self.stats(requests, self.clock() - t0)

    def stats(self, requests: List[Request], elapsed: float) -> dict:
        done = [r for r in requests if r.done >= 0]
        lat = np.array([r.latency for r in done]) if done else np.zeros(0)
        first = min((r.arrival for r in requests), default=0.0)
        last = max((r.done for r in done), default=0.0)
        span = max(last - first, 1e-9)
        return {
            "requests": len(requests), "completed": len(done), "elapsed_s": elapsed,
            "solves_per_s": len(done) / span if done else 0.0,
            "p50_latency_s": float(np.percentile(lat, 50)) if done else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if done else None,
            "mean_iterations": float(np.mean([r.iterations for r in done])) if done else None,
            "node_iterations": float(sum(r.nodes * r.iterations for r in done)),
            "cohorts": self.n_cohorts, "peak_bytes": self.peak_in_use, "budget_bytes": self.budget,
            "rejected": len(self.rejected),
        }


def loader_pool(n_threads: int, initializer: Optional[Callable] = None, initargs=(), timeout: float = 60.0):
    """A thread pool for ``Server(loader=pool.submit)`` whose threads all
    exist, each past ``initializer(*initargs)`` (e.g. selecting the device),
    when it is returned.  A pool thread that starts later, while the
    scheduling loop is capturing a cohort's CUDA graph, can invalidate that
    capture with its first CUDA calls.  The caller shuts the pool down (or
    uses it as a context manager)."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    n = max(1, int(n_threads))
    pool = ThreadPoolExecutor(max_workers=n, initializer=initializer, initargs=tuple(initargs))
    gate = threading.Barrier(n)
    try:
        # n tasks that wait for one another can only finish on n threads
        list(pool.map(lambda _: gate.wait(timeout=timeout), range(n)))
    except BaseException:
        pool.shutdown(wait=False)
        raise
    return pool


def serve_one_at_a_time(solver_factory: Callable, requests: List[Request], round_iters: int = 64,
                        variant: str = "dcfr", target_rel: float = 1e-3, clock=time.perf_counter,
                        time_limit: float = float("inf"), max_iterations: int = 100000) -> dict:
    """The baseline: one request at a time in arrival order, each loaded alone
    and iterated in rounds until it meets its target."""
    pending = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    for r in pending:
        now = clock() - t0
        if now > time_limit:
            break
        while clock() - t0 < r.arrival:
            if clock is time.perf_counter:
                time.sleep(min(r.arrival - (clock() - t0), 1e-3) if r.arrival > clock() - t0 else 0)
        s = solver_factory([r.tree], None)
        r.admitted = clock() - t0
        it = 0
        while True:
            s.iterate(round_iters, variant)
            it += round_iters
            e, _, _ = s.exploitability_batch()
            if e[0] <= target_rel * r.payoff_range or it >= max_iterations:
                break
        r.iterations = it
        r.done = clock() - t0
        s.close()
    srv = Server(solver_factory)
    return srv.stats(requests, clock() - t0)
