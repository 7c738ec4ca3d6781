"""Serving loop with continuous batching: subgame-solve requests admitted
as memory frees up and iterated until each meets its exploitability target.

Requests arrive over time (each a game tree).  The loop:

* admits the requests that have arrived into a new *cohort* (one batched
  context on its own CUDA stream) while their estimated device bytes fit the
  budget, compiling and uploading it on a loader thread;
* runs every live cohort in rounds of K iterations with its solved games
  masked off; a round queues the iterations and the FP64 exploitability of
  every game on the cohort's stream, and the loop polls each round's event,
  so cohorts never wait for one another;
* completes a game at or below ``target_rel`` x (max payoff - min payoff),
  recording completion - arrival as the request's latency;
* returns memory as games finish, not as cohorts finish: the unfinished
  games of a cohort that is mostly solved join the next new cohort, their
  state moved exactly between contexts (``copy_states_from``) at a round
  boundary, and the old context is freed.  A game's iterations are the same
  alone, in a cohort or moved between cohorts (every launch computes each
  game as it would alone).

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
    exploitability: float = float("nan")   # at completion
    moves: int = 0                          # times moved to a new cohort

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
    def __init__(self, reqs: List[Request], est_bytes: float):
        self.reqs = reqs
        self.solver = None
        self.active = np.ones(len(reqs), dtype=np.uint8)
        self.bytes = est_bytes
        self.round = None          # the round in flight (start_round's handle)
        self.moving_to = None      # the cohort its unfinished games move into
        self.sources = []          # cohorts whose unfinished games move into this one: (cohort, [(dst, src)])
        self.started = False

    @property
    def finished(self) -> bool:
        return not self.active.any()

    def live_nodes(self) -> int:
        return sum(r.nodes for r, a in zip(self.reqs, self.active) if a)


class Server:
    """`solver_factory(trees, stream)` returns an object with the Solver
    methods start_round(n, variant, active=mask) (a handle with done() and
    result()), copy_states_from(src, dst_games, src_games), sizes() and
    close().  `stream_factory()` returns a stream per cohort."""

    def __init__(self, solver_factory: Callable, hbm_budget: float = 120e9, round_iters: int = 64,
                 variant: str = "dcfr", target_rel: float = 1e-3, bytes_per_node: float = 90.0,
                 max_cohort: int = 4096, max_cohort_nodes: float = 4e6, stream_factory: Optional[Callable] = None,
                 clock: Callable[[], float] = time.perf_counter, max_iterations: int = 100000,
                 loader: Optional[Callable] = None, repack_live: float = 0.5, on_complete: Optional[Callable] = None):
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
        # a cohort whose unfinished games hold less than this fraction of its
        # nodes moves them into the next new cohort
        self.repack_live = float(repack_live)
        # on_complete(request, solver, game index): called as a game completes
        self.on_complete = on_complete
        self.cohorts: List[Cohort] = []
        self.in_use = 0.0
        self.peak_in_use = 0.0
        self.n_cohorts = 0
        self.n_moves = 0
        self.rejected: List[Request] = []

    def estimate(self, req: Request) -> float:
        return req.nodes * self.bytes_per_node

    def _admit(self, pending: List[Request], now: float, room: float) -> List[Request]:
        """Take arrived requests, in arrival order, while they fit `room`.  A
        request larger than the whole budget can never be admitted: it is
        rejected (done stays negative, counted in the stats)."""
        take = []
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

    def _sparse(self) -> List[Cohort]:
        """Running cohorts whose unfinished games are worth moving."""
        out = []
        for c in self.cohorts:
            if c.moving_to is not None or not c.started or c.finished:
                continue
            total = sum(r.nodes for r in c.reqs)
            if c.live_nodes() < self.repack_live * total:
                out.append(c)
        return out

    def _form(self, pending: List[Request], now: float, t0: float, loading: list) -> bool:
        """Form one new cohort from arrived requests and the unfinished games
        of sparse cohorts; returns False when there is nothing to form."""
        sparse = self._sparse()
        movers = [(c, k) for c in sparse for k in range(len(c.reqs)) if c.active[k]]
        room = self.budget - self.in_use - sum(self.estimate(c.reqs[k]) for c, k in movers)
        take = self._admit(pending, now, room)
        waiting = bool(pending) and pending[0].arrival <= now
        if not take and not (movers and waiting):
            # nothing arrived that fits; unfinished games move on their own
            # only when that frees memory for a request that is waiting
            return False
        reqs = take + [c.reqs[k] for c, k in movers]
        if not reqs:
            return False
        c = Cohort(reqs, sum(self.estimate(r) for r in reqs))
        self.in_use += c.bytes
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        self.n_cohorts += 1
        for src in sparse:
            pairs = [(len(take) + i, k) for i, (s_, k) in enumerate(movers) if s_ is src]
            if pairs:
                src.moving_to = c
                c.sources.append((src, pairs))
        trees, stream = [r.tree for r in reqs], self.stream_factory()
        if self.loader is None:
            c.solver = self.factory(trees, stream)
            self._ready(c, t0)
        else:
            loading.append((self.loader(lambda ts=trees, st=stream: self.factory(ts, st)), c))
        return True

    def _ready(self, c: Cohort, t0: float):
        """A loaded cohort joins the loop; its bytes are re-counted from what
        the library really holds."""
        real = float(c.solver.sizes()["device_bytes"])
        self.bytes_per_node = max(self.bytes_per_node, real / max(1, sum(r.nodes for r in c.reqs)))
        self.in_use += max(real, c.bytes) - c.bytes
        c.bytes = max(real, c.bytes)
        self.peak_in_use = max(self.peak_in_use, self.in_use)
        now = self.clock() - t0
        for r in c.reqs:
            if r.admitted < 0:
                r.admitted = now
        self.cohorts.append(c)

    def _move_in(self, c: Cohort) -> bool:
        """Take the unfinished games of c's source cohorts once each is between
        rounds; frees a source once its games are in.  True when c may run."""
        for src, pairs in list(c.sources):
            if src.round is not None:
                continue
            live = [(d, k) for d, k in pairs if src.active[k]]
            for d, k in pairs:
                if not src.active[k]:
                    c.active[d] = 0     # solved in the meantime (its slot idles)
            if live:
                c.solver.copy_states_from(src.solver, [d for d, _ in live], [k for _, k in live])
                for d, k in live:
                    src.active[k] = 0
                    c.reqs[d].moves += 1
                self.n_moves += len(live)
            c.sources.remove((src, pairs))
            if src.finished:
                self._free(src)
        return not c.sources

    def _free(self, c: Cohort):
        c.solver.close()
        self.in_use -= c.bytes
        self.cohorts.remove(c)

    def _complete(self, c: Cohort, expl: np.ndarray, now: float):
        for k, r in enumerate(c.reqs):
            if not c.active[k]:
                continue
            r.iterations += self.round_iters
            r.exploitability = float(expl[k])
            if expl[k] <= self.target_rel * r.payoff_range or r.iterations >= self.max_iterations:
                c.active[k] = 0
                r.done = now
                if self.on_complete is not None:
                    self.on_complete(r, c.solver, k)

    def run(self, requests: List[Request], time_limit: float = float("inf")) -> dict:
        pending = sorted(requests, key=lambda r: r.arrival)
        loading = []   # (future, cohort without solver)
        t0 = self.clock()
        while pending or self.cohorts or loading:
            now = self.clock() - t0
            if now > time_limit:
                break
            progress = False
            while self._form(pending, now, t0, loading):
                progress = True
            for item in [x for x in loading if x[0].done()]:
                loading.remove(item)
                item[1].solver = item[0].result()
                self._ready(item[1], t0)
                progress = True
            for c in list(self.cohorts):
                if c not in self.cohorts:   # freed as a source earlier in this pass
                    continue
                if not c.started:
                    if not self._move_in(c):
                        continue
                    c.started = True
                    if c.finished:      # every game was solved before it moved
                        self._free(c)
                        continue
                if c.round is not None and c.round.done():
                    expl = c.round.result()
                    c.round = None
                    self._complete(c, expl, self.clock() - t0)
                    progress = True
                if c.round is None:
                    if c.finished:
                        if c.moving_to is None or c.moving_to.started:
                            self._free(c)
                        continue
                    if c.moving_to is not None and c.moving_to.solver is not None:
                        continue        # its unfinished games are about to move
                    c.round = c.solver.start_round(self.round_iters, self.variant, active=c.active)
                    progress = True
            if not progress:
                if not self.cohorts and not loading and pending:
                    self._wait_until(t0, pending[0].arrival)
                elif self.clock is time.perf_counter:
                    time.sleep(5e-5)
        return self.stats(requests, self.clock() - t0)

    def _wait_until(self, t0: float, t: float):
        while True:
            left = t - (self.clock() - t0)
            if left <= 0:
                return
            if self.clock is time.perf_counter:
                time.sleep(min(left, 1e-3))

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
            "cohorts": self.n_cohorts, "moved_games": self.n_moves, "peak_bytes": self.peak_in_use,
            "budget_bytes": self.budget, "rejected": len(self.rejected),
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
        r.exploitability = float(e[0])
        r.done = clock() - t0
        s.close()
    srv = Server(solver_factory)
    return srv.stats(requests, clock() - t0)
