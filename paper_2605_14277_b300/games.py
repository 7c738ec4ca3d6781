"""Seeded synthetic two-player zero-sum extensive-form games.

This module only lays out game trees.  It holds none of the CFR arithmetic
and is the one module shared by the CUDA path and the CPU oracle: both
consume the same flat node arrays (the format of ``cfr_tree_desc`` in
``include/cfr.h``).

Tree format (nodes in an order where every parent precedes its children,
node 0 is the root):

* ``parent``      int32   parent node, -1 for the root
* ``kind``        int8    0 chance, 1 player-1 decision, 2 player-2 decision, 3 terminal
* ``infoset``     int32   decision nodes: infoset id, dense 0..J_i-1 per player; -1 otherwise
* ``action``      int32   index of the edge from the parent (0..|A|-1); -1 for the root
* ``chance_prob`` float64 probability of the edge from a chance parent, 1.0 otherwise
* ``payoff``      float64 terminal utility to player 1 (player 2 receives the negative)

Workloads (all seeded):

* ``random_game``        layered random game with chance events whose outcomes
                          each player observes only through a partition into
                          classes; infosets merge same-history nodes that differ
                          only in unobserved chance (perfect recall by
                          construction).
* ``sized_random_game``  random game aimed at a target node count.
* ``poker_game``         two-round fixed-limit poker with a 6-card deck.
* ``matrix_game``        a normal-form game written as a two-level tree.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CHANCE, P1, P2, TERMINAL = 0, 1, 2, 3


@dataclass
class Tree:
    parent: np.ndarray
    kind: np.ndarray
    infoset: np.ndarray
    action: np.ndarray
    chance_prob: np.ndarray
    payoff: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.parent = np.ascontiguousarray(self.parent, dtype=np.int32)
        self.kind = np.ascontiguousarray(self.kind, dtype=np.int8)
        self.infoset = np.ascontiguousarray(self.infoset, dtype=np.int32)
        self.action = np.ascontiguousarray(self.action, dtype=np.int32)
        self.chance_prob = np.ascontiguousarray(self.chance_prob, dtype=np.float64)
        self.payoff = np.ascontiguousarray(self.payoff, dtype=np.float64)

    @property
    def n_nodes(self) -> int:
        return int(self.parent.shape[0])

    def payoff_range(self) -> float:
        t = self.payoff[self.kind == TERMINAL]
        return float(t.max() - t.min()) if t.size else 0.0

    def n_infosets(self, player: int) -> int:
        m = self.kind == player
        return int(self.infoset[m].max()) + 1 if m.any() else 0

    def counts(self) -> dict:
        k = self.kind
        return {
            "nodes": self.n_nodes,
            "terminals": int((k == TERMINAL).sum()),
            "chance_nodes": int((k == CHANCE).sum()),
            "decision_nodes": int(((k == P1) | (k == P2)).sum()),
            "infosets_p1": self.n_infosets(P1),
            "infosets_p2": self.n_infosets(P2),
        }


def concat_trees(trees):
    """Stack several trees into one list (used to hand a batch to a loader)."""
    return list(trees)


# ----------------------------------------------------------------------------
# layered random games
# ----------------------------------------------------------------------------

def _random_partition(rng, n_outcomes, n_classes):
    """Class label per chance outcome, every class non-empty."""
    if n_classes >= n_outcomes:
        return rng.permutation(n_outcomes).astype(np.int64)
    labels = np.concatenate([np.arange(n_classes),
                             rng.integers(0, n_classes, n_outcomes - n_classes)])
    return rng.permutation(labels).astype(np.int64)


def random_game(seed: int, depth: int, chance: dict, actions=(2, 3), action_p=None,
                n_classes=2, partitions=None, payoff="normal", name="") -> Tree:
    """Layered random two-player zero-sum game with perfect recall.

    * depth: terminals sit at this depth (root is depth 0).
    * chance: {depth: number of uniform outcomes} for chance levels.
    * Decision levels alternate player 1, player 2, ... skipping chance levels.
    * Each player observes chance event e only through ``partitions[e][p]``
      (class label per outcome); all actions are public.  A player's infoset
      key is (public action history, observed classes so far), so nodes that
      differ only in unobserved chance outcomes share an infoset and all nodes
      of an infoset share the player's own history (perfect recall).
    * The action count of an infoset is drawn per infoset from ``actions``.
    * payoff: 'int2' (uniform integer in [-2, 2]), 'normal' (N(0,1) rounded to
      float32) or 'uniform' (U[-1,1] rounded to float32).
    """
    rng = np.random.default_rng(seed)
    chance_depths = sorted(chance)
    if partitions is None:
        partitions = {}
        for d in chance_depths:
            partitions[d] = {p: _random_partition(rng, chance[d], n_classes) for p in (P1, P2)}
    actions = np.asarray(actions, dtype=np.int64)
    # decision player per depth
    player_at = {}
    nxt = P1
    for d in range(depth):
        if d in chance:
            continue
        player_at[d] = nxt
        nxt = P2 if nxt == P1 else P1

    pub = np.zeros(1, dtype=np.int64)            # public history id per node at this depth
    obs = {P1: np.zeros(1, np.int64), P2: np.zeros(1, np.int64)}  # packed observed classes
    par_list, kind_list, inf_list, act_list, cp_list = [], [], [], [], []
    par = np.array([-1], dtype=np.int64)
    act = np.array([-1], dtype=np.int64)
    cp = np.array([1.0])
    base = 0
    n_inf = {P1: 0, P2: 0}
    payoff_arr = None
    for d in range(depth + 1):
        n = pub.shape[0]
        par_list.append(par)
        act_list.append(act)
        cp_list.append(cp)
        if d == depth:
            kind_list.append(np.full(n, TERMINAL, np.int8))
            inf_list.append(np.full(n, -1, np.int64))
            if payoff == "int2":
                pv = rng.integers(-2, 3, n).astype(np.float64)
            elif payoff == "normal":
                pv = rng.standard_normal(n).astype(np.float32).astype(np.float64)
            elif payoff == "uniform":
                pv = rng.uniform(-1.0, 1.0, n).astype(np.float32).astype(np.float64)
            else:
                raise ValueError(payoff)
            payoff_arr = pv
            break
        idx = np.arange(n, dtype=np.int64)
        if d in chance:
            k = chance[d]
            kind_list.append(np.full(n, CHANCE, np.int8))
            inf_list.append(np.full(n, -1, np.int64))
            nch = np.full(n, k, dtype=np.int64)
            child_par = np.repeat(idx, nch)
            child_act = np.tile(np.arange(k, dtype=np.int64), n)
            child_pub = pub[child_par]          # chance is private: public history unchanged
            new_obs = {}
            for p in (P1, P2):
                cls = partitions[d][p][child_act]
                new_obs[p] = obs[p][child_par] * 16 + cls
            obs = new_obs
            cp = np.full(child_par.shape[0], 1.0 / k)
        else:
            p = player_at[d]
            kind_list.append(np.full(n, p, np.int8))
            key = pub * 4096 + obs[p]
            uk, inv = np.unique(key, return_inverse=True)
            if action_p is None:
                na_inf = rng.choice(actions, size=uk.shape[0])
            else:
                na_inf = rng.choice(actions, size=uk.shape[0], p=action_p)
            inf_list.append(inv.astype(np.int64) + n_inf[p])
            n_inf[p] += uk.shape[0]
            nch = na_inf[inv]
            child_par = np.repeat(idx, nch)
            starts = np.cumsum(nch) - nch
            child_act = np.arange(child_par.shape[0], dtype=np.int64) - np.repeat(starts, nch)
            raw = pub[child_par] * 8 + child_act
            _, child_pub = np.unique(raw, return_inverse=True)
            obs = {q: obs[q][child_par] for q in (P1, P2)}
            cp = np.ones(child_par.shape[0])
        pub = child_pub.astype(np.int64)
        par = child_par + base
        act = child_act
        base += n
    parent = np.concatenate(par_list)
    kind = np.concatenate(kind_list)
    infoset = np.concatenate(inf_list)
    action = np.concatenate(act_list)
    cprob = np.concatenate(cp_list)
    pay = np.zeros(parent.shape[0])
    pay[parent.shape[0] - payoff_arr.shape[0]:] = payoff_arr
    meta = {"seed": seed, "depth": depth, "chance": dict(chance),
            "partitions": {d: {p: partitions[d][p].tolist() for p in (P1, P2)} for d in partitions}}
    return Tree(parent, kind, infoset, action, cprob, pay, name=name, meta=meta)


def sized_random_game(seed: int, target_nodes: float, depth_range=(4, 10), actions=(2, 4),
                      payoff="uniform", root_outcomes=(2, 3), name="") -> Tree:
    """Random game aimed at ``target_nodes`` nodes (actual count recorded in meta).

    A root chance event with 2-3 outcomes (each player sees a 2-class partition)
    is followed by ``depth`` decision levels; the per-infoset action count is a
    two-point mix of the integers around the branching factor that hits the
    target at that depth.
    """
    rng = np.random.default_rng(seed)
    k = int(rng.integers(root_outcomes[0], root_outcomes[1] + 1))
    lo_a, hi_a = actions
    dmin, dmax = depth_range

    def nodes_for(b, dd):   # 1 chance root + k * sum_{i<=dd-1} b^i decision/terminal levels
        return 1 + k * sum(b ** i for i in range(dd))

    dd = int(rng.integers(dmin, dmax + 1))
    # adjust depth so the target is reachable with branching in [lo_a, hi_a]
    while dd > dmin and nodes_for(lo_a, dd) > target_nodes:
        dd -= 1
    while dd < dmax and nodes_for(hi_a, dd) < target_nodes:
        dd += 1
    lo, hi = float(lo_a), float(hi_a)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if nodes_for(mid, dd) < target_nodes:
            lo = mid
        else:
            hi = mid
    b = min(max(0.5 * (lo + hi), lo_a), hi_a)
    fl = int(math.floor(b))
    if fl >= hi_a:
        acts, ap = (hi_a,), None
    else:
        frac = b - fl
        acts, ap = (fl, fl + 1), [1.0 - frac, frac]
    sub_seed = int(rng.integers(0, 2**31 - 1))
    t = random_game(sub_seed, depth=dd, chance={0: k}, actions=acts, action_p=ap, n_classes=2,
                    payoff=payoff, name=name)
    t.meta.update({"seed": seed, "target_nodes": float(target_nodes), "branching": b})
    return t


# ----------------------------------------------------------------------------
# the configured workloads
# ----------------------------------------------------------------------------

def small_random_game(seed: int = 1) -> Tree:
    """~400-500 nodes: root chance with 3 outcomes, depth 6, 2-3 actions,
    integer payoffs in [-2, 2]; each player sees a random 1..3-way merge of
    the chance outcomes."""
    rng = np.random.default_rng(seed + 7919)
    while True:
        a = _random_partition(rng, 3, 2)
        b = _random_partition(rng, 3, 2)
        if not np.array_equal(a, b):
            break
    parts = {0: {P1: a, P2: b}}
    return random_game(seed, depth=6, chance={0: 3}, actions=(2, 3), partitions=parts,
                       payoff="int2", name=f"small_random_d6_s{seed}")


def large_random_game(seed: int = 3) -> Tree:
    """Depth 12, 3-4 actions, chance at depths 0 and 6 (4 outcomes each), each
    player sees a 2-class partition of each chance event, N(0,1) payoffs:
    ~4.4e6 terminals, ~6.2e6 nodes."""
    return random_game(seed, depth=12, chance={0: 4, 6: 4}, actions=(3, 4), n_classes=2,
                       payoff="normal", name=f"large_random_d12_s{seed}")


def batch_games(n_games: int = 4096, seed0: int = 1000, lo: float = 1e2, hi: float = 1e5):
    """Seeded games with node counts log-uniform in [lo, hi], depth 4-10, 2-4
    actions, U[-1,1] payoffs."""
    return [batch_game(s, lo, hi) for s in range(seed0, seed0 + n_games)]


def batch_game(seed: int, lo: float = 1e2, hi: float = 1e5) -> Tree:
    """Game `seed` of the batched workload (see batch_games)."""
    rng = np.random.default_rng(seed)
    target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
    return sized_random_game(seed, target, depth_range=(4, 10), actions=(2, 4),
                             payoff="uniform", name=f"batch_s{seed}")


def batch_sample_seeds(n_sample: int = 64, n_games: int = 4096, seed0: int = 1000):
    """Seeds of an evenly spaced sample of the batched workload's games."""
    step = max(1, n_games // n_sample)
    return [seed0 + k * step for k in range(n_sample)]


def serving_request(seed: int, lo: float = 1e3, hi: float = 1e6) -> Tree:
    """One subgame-solve request: nodes log-uniform in [lo, hi], N(0,1) payoffs."""
    rng = np.random.default_rng(seed)
    target = math.exp(rng.uniform(math.log(lo), math.log(hi)))
    return sized_random_game(seed, target, depth_range=(4, 10), actions=(2, 4),
                             payoff="normal", name=f"req_s{seed}")


def poisson_arrivals(seed: int, rate: float, n: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: seeded exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


# ----------------------------------------------------------------------------
# poker: 6-card deck (3 ranks x 2 suits), one private card each, one public
# card after round one, ante 1, fixed bets 2 then 4, at most 2 bets/raises per
# round, a pair with the public card beats any high card.
# ----------------------------------------------------------------------------

FOLD, CALL, RAISE = 0, 1, 2


def poker_game(n_ranks: int = 3, n_suits: int = 2, ante: float = 1.0, bets=(2.0, 4.0),
               raise_cap: int = 2, name="poker_6card_2round") -> Tree:
    cards = [(r, s) for r in range(n_ranks) for s in range(n_suits)]
    parent, kind, infoset, action, cprob, payoff = [], [], [], [], [], []
    inf_ids = {P1: {}, P2: {}}
    # breadth-first construction: queue of (node_id, state)
    from collections import deque

    def new_node(par, k, act, prob):
        parent.append(par)
        kind.append(k)
        infoset.append(-1)
        action.append(act)
        cprob.append(prob)
        payoff.append(0.0)
        return len(parent) - 1

    def showdown(c1, c2, pub):
        r1, r2, rp = cards[c1][0], cards[c2][0], cards[pub][0]
        s1 = (1, r1) if r1 == rp else (0, r1)
        s2 = (1, r2) if r2 == rp else (0, r2)
        return (s1 > s2) - (s1 < s2)

    root = new_node(-1, CHANCE, -1, 1.0)
    q = deque()
    q.append((root, ("deal1",)))
    while q:
        nid, st = q.popleft()
        tag = st[0]
        if tag == "deal1":
            for i, c in enumerate(range(len(cards))):
                ch = new_node(nid, CHANCE, i, 1.0 / len(cards))
                q.append((ch, ("deal2", c)))
        elif tag == "deal2":
            c1 = st[1]
            rest = [c for c in range(len(cards)) if c != c1]
            for i, c in enumerate(rest):
                # player 1 opens round 1
                ch = new_node(nid, P1, i, 1.0 / len(rest))
                q.append((ch, ("bet", c1, c, None, 0, "", [ante, ante], 0, 0)))
        elif tag == "public":
            _, c1, c2, hist, contrib = st
            rest = [c for c in range(len(cards)) if c not in (c1, c2)]
            kind[nid] = CHANCE
            for i, c in enumerate(rest):
                ch = new_node(nid, P1, i, 1.0 / len(rest))
                q.append((ch, ("bet", c1, c2, c, 1, hist + "/", list(contrib), 0, 0)))
        elif tag == "bet":
            _, c1, c2, pub, rnd, hist, contrib, n_raises, n_acts = st
            p = P1 if (n_acts % 2 == 0) else P2
            me, op = (0, 1) if p == P1 else (1, 0)
            facing = contrib[op] > contrib[me]
            legal = []
            if facing:
                legal.append(FOLD)
            legal.append(CALL)
            if n_raises < raise_cap:
                legal.append(RAISE)
            priv = c1 if p == P1 else c2
            key = (priv, pub, hist)
            d = inf_ids[p]
            if key not in d:
                d[key] = len(d)
            infoset[nid] = d[key]
            kind[nid] = p
            for i, a in enumerate(legal):
                if a == FOLD:
                    ch = new_node(nid, TERMINAL, i, 1.0)
                    payoff[ch] = -contrib[0] if p == P1 else contrib[1]
                elif a == CALL:
                    c = list(contrib)
                    c[me] = c[op]
                    closes = facing or n_acts >= 1
                    h = hist + "c"
                    if closes:
                        if rnd == 0:
                            ch = new_node(nid, CHANCE, i, 1.0)
                            q.append((ch, ("public", c1, c2, h, c)))
                        else:
                            ch = new_node(nid, TERMINAL, i, 1.0)
                            w = showdown(c1, c2, pub)
                            payoff[ch] = c[1] if w > 0 else (-c[0] if w < 0 else 0.0)
                    else:
                        ch = new_node(nid, P2 if p == P1 else P1, i, 1.0)
                        q.append((ch, ("bet", c1, c2, pub, rnd, h, c, n_raises, n_acts + 1)))
                else:
                    c = list(contrib)
                    c[me] = c[op] + bets[rnd]
                    ch = new_node(nid, P2 if p == P1 else P1, i, 1.0)
                    q.append((ch, ("bet", c1, c2, pub, rnd, hist + "r", c, n_raises + 1, n_acts + 1)))
    # the breadth-first queue visits parents before children, so ids already satisfy
    # parent < child
    return Tree(np.array(parent), np.array(kind), np.array(infoset), np.array(action),
                np.array(cprob), np.array(payoff), name=name,
                meta={"ranks": n_ranks, "suits": n_suits, "ante": ante, "bets": list(bets),
                      "raise_cap": raise_cap})


# ----------------------------------------------------------------------------
# normal-form games
# ----------------------------------------------------------------------------

def matrix_game(A, name="matrix") -> Tree:
    """Player 1 picks a row, player 2 (not seeing it) a column; payoff A[i,j] to player 1."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    parent = [-1]
    kind = [P1]
    infoset = [0]
    action = [-1]
    for i in range(m):
        parent.append(0)
        kind.append(P2)
        infoset.append(0)
        action.append(i)
    pay = [0.0] * (m + 1)
    for i in range(m):
        for j in range(n):
            parent.append(1 + i)
            kind.append(TERMINAL)
            infoset.append(-1)
            action.append(j)
            pay.append(A[i, j])
    N = len(parent)
    return Tree(np.array(parent), np.array(kind), np.array(infoset), np.array(action),
                np.ones(N), np.array(pay), name=name, meta={"A": A.tolist()})


def rps() -> Tree:
    return matrix_game([[0, -1, 1], [1, 0, -1], [-1, 1, 0]], name="rps")


def random_2x2_no_saddle(seed: int):
    """Seeded 2x2 integer matrix without a pure-strategy saddle point."""
    rng = np.random.default_rng(seed)
    while True:
        A = rng.integers(-5, 6, (2, 2)).astype(np.float64)
        saddle = False
        for i in range(2):
            for j in range(2):
                if A[i, j] == A[i, :].min() and A[i, j] == A[:, j].max():
                    saddle = True
        den = A[0, 0] - A[0, 1] - A[1, 0] + A[1, 1]
        if not saddle and den != 0:
            return A


def random_fully_mixed(seed: int, n: int):
    """n x n matrix whose unique equilibrium (p*, q*, v) is fully mixed.

    Start from a random matrix and remove the components that keep p* and q*
    from equalising: C q* = v 1 and p*^T C = v 1^T.
    """
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.5, 1.5, n)
    p /= p.sum()
    qv = rng.uniform(0.5, 1.5, n)
    qv /= qv.sum()
    v = float(rng.uniform(-1, 1))
    B = rng.standard_normal((n, n))
    ones = np.ones(n)
    A = B - np.outer(B @ qv - v * ones, qv) / (qv @ qv)
    C = A - np.outer(p, p @ A - v * ones) / (p @ p)
    return C, p, qv, v


# ----------------------------------------------------------------------------
# n-player games (payoff tensors)
# ----------------------------------------------------------------------------
#
# Tree format of ``cfrn_tree_desc`` in include/cfr_nplayer.h (nodes in an order
# where every parent precedes its children, node 0 is the root):
#
# * ``parent``      int32   parent node, -1 for the root
# * ``kind``        int8    0 chance, 1 decision, 2 terminal
# * ``actor``       int8    decision nodes: the acting player 0..n-1; -1 otherwise
# * ``infoset``     int32   decision nodes: infoset id, dense 0..J_i-1 per player; -1 otherwise
# * ``action``      int32   index of the edge from the parent (0..|A|-1); -1 for the root
# * ``chance_prob`` float64 probability of the edge from a chance parent, 1.0 otherwise
# * ``payoff``      float64 [n_nodes, n_players] terminal utilities (0 elsewhere)

N_CHANCE, N_DECISION, N_TERMINAL = 0, 1, 2


@dataclass
class NTree:
    n_players: int
    parent: np.ndarray
    kind: np.ndarray
    actor: np.ndarray
    infoset: np.ndarray
    action: np.ndarray
    chance_prob: np.ndarray
    payoff: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.parent = np.ascontiguousarray(self.parent, dtype=np.int32)
        self.kind = np.ascontiguousarray(self.kind, dtype=np.int8)
        self.actor = np.ascontiguousarray(self.actor, dtype=np.int8)
        self.infoset = np.ascontiguousarray(self.infoset, dtype=np.int32)
        self.action = np.ascontiguousarray(self.action, dtype=np.int32)
        self.chance_prob = np.ascontiguousarray(self.chance_prob, dtype=np.float64)
        self.payoff = np.ascontiguousarray(self.payoff, dtype=np.float64).reshape(-1, self.n_players)

    @property
    def n_nodes(self) -> int:
        return int(self.parent.shape[0])

    def n_infosets(self, player: int) -> int:
        m = (self.kind == N_DECISION) & (self.actor == player)
        return int(self.infoset[m].max()) + 1 if m.any() else 0

    def payoff_range(self) -> float:
        t = self.payoff[self.kind == N_TERMINAL]
        return float(t.max() - t.min()) if t.size else 0.0

    def counts(self) -> dict:
        k = self.kind
        out = {"nodes": self.n_nodes, "players": self.n_players, "terminals": int((k == N_TERMINAL).sum()),
               "chance_nodes": int((k == N_CHANCE).sum()), "decision_nodes": int((k == N_DECISION).sum())}
        for p in range(self.n_players):
            out[f"infosets_{p}"] = self.n_infosets(p)
        return out


def nplayer_from_two_player(tree: Tree, n_players: int = 2) -> NTree:
    """The two-player tree in the n-player format: player 1 is player 0,
    player 2 is player 1 (payoff -u1); any further players never act and
    receive 0 (their only sequence is the empty one)."""
    if n_players < 2:
        raise ValueError("n_players >= 2")
    k = tree.kind
    kind = np.where(k == CHANCE, N_CHANCE, np.where(k == TERMINAL, N_TERMINAL, N_DECISION)).astype(np.int8)
    actor = np.where(k == P1, 0, np.where(k == P2, 1, -1)).astype(np.int8)
    pay = np.zeros((tree.n_nodes, n_players))
    term = k == TERMINAL
    pay[term, 0] = tree.payoff[term]
    pay[term, 1] = -tree.payoff[term]
    return NTree(n_players, tree.parent, kind, actor, tree.infoset, tree.action, tree.chance_prob, pay,
                 name=(tree.name or "game") + f"_as_{n_players}p", meta=dict(tree.meta))


def random_nplayer_game(n_players: int, seed: int, depth: int, chance: dict, actions=(2, 3),
                        n_classes=2, payoff="normal", zero_sum=True, name="") -> NTree:
    """Layered random n-player game with perfect recall (the n-player form of
    ``random_game``): decision levels cycle players 0, 1, ..., n-1, skipping
    chance levels; each player observes chance event e only through its own
    partition of the outcomes into classes; all actions are public, and a
    player's infoset key is (public history, its observed classes).

    payoff: 'normal' (N(0,1) rounded to float32) or 'int2' (integers in
    [-2, 2]) per player; zero_sum: the last player receives minus the sum of
    the others' payoffs."""
    rng = np.random.default_rng(seed)
    n = n_players
    partitions = {d: [_random_partition(rng, chance[d], n_classes) for _ in range(n)] for d in sorted(chance)}
    actions = np.asarray(actions, dtype=np.int64)
    actor_at, nxt = {}, 0
    for d in range(depth):
        if d in chance:
            continue
        actor_at[d] = nxt
        nxt = (nxt + 1) % n
    pub = np.zeros(1, dtype=np.int64)
    obs = [np.zeros(1, np.int64) for _ in range(n)]
    par_l, kind_l, act_l, inf_l, edge_l, cp_l = [], [], [], [], [], []
    par = np.array([-1], dtype=np.int64)
    edge = np.array([-1], dtype=np.int64)
    cp = np.array([1.0])
    base = 0
    n_inf = [0] * n
    term_pay = None
    for d in range(depth + 1):
        m = pub.shape[0]
        par_l.append(par)
        edge_l.append(edge)
        cp_l.append(cp)
        if d == depth:
            kind_l.append(np.full(m, N_TERMINAL, np.int8))
            act_l.append(np.full(m, -1, np.int8))
            inf_l.append(np.full(m, -1, np.int64))
            if payoff == "normal":
                pv = rng.standard_normal((m, n)).astype(np.float32).astype(np.float64)
            elif payoff == "int2":
                pv = rng.integers(-2, 3, (m, n)).astype(np.float64)
            else:
                raise ValueError(payoff)
            if zero_sum:
                pv[:, n - 1] = -pv[:, : n - 1].sum(axis=1)
            term_pay = pv
            break
        idx = np.arange(m, dtype=np.int64)
        if d in chance:
            k = chance[d]
            kind_l.append(np.full(m, N_CHANCE, np.int8))
            act_l.append(np.full(m, -1, np.int8))
            inf_l.append(np.full(m, -1, np.int64))
            cpar = np.repeat(idx, k)
            cedge = np.tile(np.arange(k, dtype=np.int64), m)
            cpub = pub[cpar]
            obs = [obs[q][cpar] * 16 + partitions[d][q][cedge] for q in range(n)]
            cp = np.full(cpar.shape[0], 1.0 / k)
        else:
            p = actor_at[d]
            kind_l.append(np.full(m, N_DECISION, np.int8))
            act_l.append(np.full(m, p, np.int8))
            key = pub * 4096 + obs[p]
            uk, inv = np.unique(key, return_inverse=True)
            na_inf = rng.choice(actions, size=uk.shape[0])
            inf_l.append(inv.astype(np.int64) + n_inf[p])
            n_inf[p] += uk.shape[0]
            nch = na_inf[inv]
            cpar = np.repeat(idx, nch)
            starts = np.cumsum(nch) - nch
            cedge = np.arange(cpar.shape[0], dtype=np.int64) - np.repeat(starts, nch)
            _, cpub = np.unique(pub[cpar] * 8 + cedge, return_inverse=True)
            obs = [obs[q][cpar] for q in range(n)]
            cp = np.ones(cpar.shape[0])
        pub = cpub.astype(np.int64)
        par = cpar + base
        edge = cedge
        base += m
    parent = np.concatenate(par_l)
    pay = np.zeros((parent.shape[0], n))
    pay[parent.shape[0] - term_pay.shape[0]:] = term_pay
    meta = {"seed": seed, "depth": depth, "chance": dict(chance), "players": n}
    return NTree(n, parent, np.concatenate(kind_l), np.concatenate(act_l), np.concatenate(inf_l),
                 np.concatenate(edge_l), np.concatenate(cp_l), pay, name=name, meta=meta)


def small_nplayer_game(n_players: int = 3, seed: int = 1) -> NTree:
    """A few hundred nodes: the size the oracle runs in well under a second."""
    return random_nplayer_game(n_players, seed, depth=2 * n_players, chance={0: 3}, actions=(2, 3),
                               name=f"small_{n_players}p_s{seed}")


def large_nplayer_game(n_players: int = 3, seed: int = 5) -> NTree:
    """4.84M nodes (3 players): a chance deal of 8 outcomes that each player
    observes through its own partition into 4 classes, then 14 decision
    levels of 2-3 actions with the players in turn, and 2.9M terminals with
    zero-sum N(0,1) payoffs."""
    return random_nplayer_game(n_players, seed, depth=15, chance={0: 8}, actions=(2, 3), n_classes=4,
                               name=f"large_{n_players}p_s{seed}")


def kuhn3_game(ante: float = 1.0, bet: float = 1.0) -> NTree:
    """Three-player Kuhn poker: a deck of four ranked cards, one dealt to each
    player (24 equally likely deals), antes of 1, one betting round in seat
    order.  Before any bet a player checks (action 0) or bets 1 (action 1);
    after a bet every other player still to respond, in seat order from the
    bettor, folds (0) or calls (1).  Among the players who did not fold, the
    highest card takes the pot.  A player's infoset is its card and the public
    action history."""
    n = 3
    parent, kind, actor, infoset, action, cprob, pay = [], [], [], [], [], [], []
    inf_ids = [dict() for _ in range(n)]

    def new_node(par, k, who, act, prob):
        parent.append(par)
        kind.append(k)
        actor.append(who)
        infoset.append(-1)
        action.append(act)
        cprob.append(prob)
        pay.append([0.0] * n)
        return len(parent) - 1

    deals = [(a, b, c) for a in range(4) for b in range(4) for c in range(4) if len({a, b, c}) == 3]
    root = new_node(-1, N_CHANCE, -1, -1, 1.0)

    def play(node_par, act, cards, hist, bettor, responded, folded):
        # hist: public actions so far; bettor: seat that bet (or -1);
        # responded: seats that answered the bet
        if bettor < 0:
            seat = len(hist)
            if seat == n:   # everyone checked: showdown for the antes
                return showdown(node_par, act, cards, -1, set())
        else:
            order = [(bettor + k) % n for k in range(1, n)]
            todo = [s for s in order if s not in responded]
            if not todo:
                return showdown(node_par, act, cards, bettor, folded)
            seat = todo[0]
        node = new_node(node_par, N_DECISION, seat, act, 1.0)
        key = (cards[seat], tuple(hist))
        ids = inf_ids[seat]
        if key not in ids:
            ids[key] = len(ids)
        infoset[node] = ids[key]
        for a in (0, 1):
            if bettor < 0:
                play(node, a, cards, hist + [a], seat if a == 1 else -1, set(), set())
            else:
                play(node, a, cards, hist + [a], bettor, responded | {seat},
                     folded | ({seat} if a == 0 else set()))
        return node

    def showdown(node_par, act, cards, bettor, folded):
        node = new_node(node_par, N_TERMINAL, -1, act, 1.0)
        contrib = [ante] * n
        if bettor >= 0:
            contrib[bettor] += bet
            for s in range(n):
                if s != bettor and s not in folded:
                    contrib[s] += bet
        live = [s for s in range(n) if s not in folded]
        win = max(live, key=lambda s: cards[s])
        pot = sum(contrib)
        pay[node] = [(pot if s == win else 0.0) - contrib[s] for s in range(n)]
        return node

    for k, cards in enumerate(deals):
        play(root, k, cards, [], -1, set(), set())
    # the deal's children carry its probability
    cp = np.asarray(cprob)
    par = np.asarray(parent)
    cp[par == root] = 1.0 / len(deals)
    return NTree(n, par, kind, actor, infoset, action, cp, np.asarray(pay), name="kuhn3")


def nplayer_normal_form(tensors, name="normal_form") -> NTree:
    """An n-player normal-form game as a tree: player 0 moves, then player 1
    without seeing player 0's action, ..., each player with one infoset;
    tensors[i][a_0, ..., a_{n-1}] is player i's payoff."""
    tensors = [np.asarray(t, dtype=np.float64) for t in tensors]
    n = len(tensors)
    shape = tensors[0].shape
    parent, kind, actor, infoset, action = [-1], [N_DECISION], [0], [0], [-1]
    frontier = [(0, ())]
    for p in range(n):
        nxt = []
        for node, hist in frontier:
            for a in range(shape[p]):
                parent.append(node)
                action.append(a)
                last = p == n - 1
                kind.append(N_TERMINAL if last else N_DECISION)
                actor.append(-1 if last else p + 1)
                infoset.append(-1 if last else 0)
                nxt.append((len(parent) - 1, hist + (a,)))
        frontier = nxt
    pay = np.zeros((len(parent), n))
    for node, hist in frontier:
        pay[node] = [t[hist] for t in tensors]
    return NTree(n, np.asarray(parent), np.asarray(kind), np.asarray(actor), np.asarray(infoset),
                 np.asarray(action), np.ones(len(parent)), pay, name=name)
