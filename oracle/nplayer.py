"""Plain FP64 CPU oracle for n-player sequence-form CFR -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline and
reference legs use this module; the library never does.  It shares no code
with the CUDA path (its own tree parsing, its own sequence numbering, its own
loops) and nothing with ``oracle/cfr_oracle.c`` either.

What it computes ("Parallelizing Counterfactual Regret Minimization", Kim &
Sandholm), for a game of n >= 2 players:

* sequence form (Sec. 2.1): each player i has its own TFSDP; sequences
  sigma = (j, a) of its decision points j, the empty sequence 0, the parent
  sequence p_j of j.  Sequences are numbered in the caller's order:
  sigma(j, a) = 1 + (actions of the infosets before j) + a.
* utilities (Sec. 2.1, "tensor operations in multiplayer settings"): the
  payoff tensor of player i contracted with every other player's sequence-form
  strategy,
      u_i[s] = sum over terminals z with seq_i(z) = s of
               pi_c(z) * payoff_i(z) * prod_{k != i} x_k[seq_k(z)],
  one pass over the terminal list.
* NextStrategy (Alg. 1): regret matching b_j = (r_j)^+ / ||(r_j)^+||_1, uniform
  when the norm is 0, then x[0] = 1 and x[(j, a)] = x[p_j] b_j[a] top-down.
* ObserveUtility (Alg. 1): bottom-up counterfactual values
  V[(j, a)] = u[(j, a)] + sum of ev_j' over the decision points j' with
  p_j' = (j, a), ev_j = sum_a b_j[a] V[(j, a)], then r_j += V[(j, .)] - ev_j.
  Decision points are visited level by level (all of a level's children are
  one level deeper), which is the order of Alg. 2's bottom-up loop.
* the variants' post-ops: CFR+ (Alg. 3) r := r^+; DCFR (Alg. 4) positive
  regrets times t^alpha / (t^alpha + 1), negative ones times
  t^beta / (t^beta + 1); PCFR+ and PCFR (Alg. 5): NextStrategy*(m) with the
  prediction m = the utility just observed (back up r, keep b^(t-1),
  ObserveUtility(m), regret matching, restore r), floored as CFR+ for PCFR+,
  never floored for PCFR.
* schedules (Sec. 3.5.1): alternating -- players update in the order
  0, 1, ..., n-1, each seeing the strategies the players before it have just
  recomputed -- or simultaneous (every utility from the iteration's start).
* average strategy: xbar_i += t^gamma x_i^t for the strategy x_i^t that player
  i played at iteration t.
* NashConv (the n-player form of the exploitability that Sec. 4 reports):
  sum over players of (value of a best response to the others' normalised
  averages - value of its own normalised average against them); with two
  zero-sum players it equals twice the exploitability (BR1 + BR2) / 2.
"""
from __future__ import annotations

import numpy as np

CFR, CFR_PLUS, DCFR, PCFR_PLUS, PCFR = 0, 1, 2, 3, 4
CHANCE, DECISION, TERMINAL = 0, 1, 2


class PlayerSF:
    """One player's sequence form in the caller's numbering (index 0 = empty)."""

    def __init__(self, J, nact, par):
        self.J = int(J)
        self.nact = np.asarray(nact, dtype=np.int64)
        self.par = np.asarray(par, dtype=np.int64)            # parent sequence p_j
        self.off = 1 + np.concatenate([[0], np.cumsum(self.nact)[:-1]]) if J else np.zeros(0, np.int64)
        self.S = int(self.nact.sum())                          # non-empty sequences
        self.seq_inf = np.repeat(np.arange(J), self.nact)      # infoset of sequence 1..S
        # level of each decision point: 0 when p_j is empty, else one below
        # the level of the decision point owning p_j
        # (a fixed point: each round settles one more level)
        owner = np.concatenate([[0], self.seq_inf])[self.par]       # decision point owning p_j
        level = np.zeros(J, np.int64)
        for _ in range(J + 1):
            new = np.where(self.par == 0, 0, level[owner] + 1)
            if np.array_equal(new, level):
                break
            level = new
        else:
            raise ValueError("decision points not reachable from the empty sequence")
        self.level = level
        self.levels = [np.flatnonzero(level == d) for d in range(int(level.max()) + 1)] if J else []

    def seqs_of(self, js):
        """the sequences of decision points js, in order"""
        if len(js) == 0:
            return np.zeros(0, np.int64)
        na = self.nact[js]
        start = np.repeat(self.off[js], na)
        a = np.arange(int(na.sum())) - np.repeat(np.cumsum(na) - na, na)
        return start + a


class NGame:
    """An n-player game parsed into per-player sequence forms and a terminal list."""

    def __init__(self, tree):
        n = int(tree.n_players)
        parent = np.asarray(tree.parent, np.int64)
        kind = np.asarray(tree.kind, np.int64)
        actor = np.asarray(tree.actor, np.int64)
        infoset = np.asarray(tree.infoset, np.int64)
        action = np.asarray(tree.action, np.int64)
        cprob = np.asarray(tree.chance_prob, np.float64)
        payoff = np.asarray(tree.payoff, np.float64).reshape(-1, n)
        N = parent.shape[0]
        self.n = n
        # depth of every node (parents precede children)
        depth = np.zeros(N, np.int64)
        for _ in range(N):
            nd = np.where(parent < 0, 0, depth[np.maximum(parent, 0)] + 1)
            if np.array_equal(nd, depth):
                break
            depth = nd
        # action counts per infoset: children of one node of the infoset
        nch = np.bincount(parent[1:], minlength=N) if N > 1 else np.zeros(N, np.int64)
        self.pl = []
        for p in range(n):
            dm = (kind == DECISION) & (actor == p)
            J = int(infoset[dm].max()) + 1 if dm.any() else 0
            nact = np.zeros(J, np.int64)
            nact[infoset[dm]] = nch[dm]
            self.pl.append([J, nact])
        offs = [1 + np.concatenate([[0], np.cumsum(nact)[:-1]]) if J else np.zeros(0, np.int64)
                for J, nact in self.pl]
        # each node's current sequence of every player, level by level
        seq = np.zeros((N, n), np.int64)
        reach = np.ones(N)
        for d in range(1, int(depth.max()) + 1 if N else 0):
            idx = np.flatnonzero(depth == d)
            par = parent[idx]
            seq[idx] = seq[par]
            pk = kind[par]
            dec = pk == DECISION
            for p in range(n):
                m = dec & (actor[par] == p)
                seq[idx[m], p] = offs[p][infoset[par[m]]] + action[idx[m]]
            reach[idx] = reach[par] * np.where(pk == CHANCE, cprob[idx], 1.0)
        # parent sequence of every infoset (perfect recall: one per infoset)
        players = []
        for p in range(n):
            J, nact = self.pl[p]
            dm = np.flatnonzero((kind == DECISION) & (actor == p))
            par = np.full(J, -1, np.int64)
            par[infoset[dm]] = seq[dm, p]
            if J and (par[infoset[dm]] != seq[dm, p]).any():
                raise ValueError(f"player {p}: nodes of one infoset differ in the player's own history")
            players.append(PlayerSF(J, nact, par))
        self.pl = players
        term = np.flatnonzero(kind == TERMINAL)
        self.tseq = seq[term]                  # [Z, n] sequences of the terminals
        self.treach = reach[term]              # pi_c(z)
        self.tpay = payoff[term]               # [Z, n]

    # ---- the steps ------------------------------------------------------
    def utility(self, i, xs):
        """u_i = player i's payoff tensor contracted with the others' x (Sec. 2.1)"""
        prod = self.treach * self.tpay[:, i]
        for k in range(self.n):
            if k != i:
                prod = prod * xs[k][self.tseq[:, k]]
        u = np.zeros(self.pl[i].S + 1)
        np.add.at(u, self.tseq[:, i], prod)
        return u

    @staticmethod
    def regret_matching(P, r):
        """NextStrategy, first half (Alg. 1)"""
        q = np.maximum(r[1:], 0.0)
        b = np.zeros(P.S + 1)
        if P.J == 0:
            return b
        s = np.add.reduceat(q, P.off - 1)
        sj = s[P.seq_inf]
        b[1:] = np.where(sj > 0.0, q / np.where(sj > 0.0, sj, 1.0), 1.0 / P.nact[P.seq_inf])
        return b

    @staticmethod
    def sequence_form(P, b):
        """NextStrategy, second half (Alg. 1): x[0] = 1, top-down"""
        x = np.zeros(P.S + 1)
        x[0] = 1.0
        for js in P.levels:
            ss = P.seqs_of(js)
            x[ss] = x[P.par[P.seq_inf[ss - 1]]] * b[ss]
        return x

    @staticmethod
    def observe_utility(P, u, b, r):
        """ObserveUtility (Alg. 1): V and ev bottom-up, then r += V - ev (in place)"""
        V = u.copy()
        ev = np.zeros(P.J)
        for js in reversed(P.levels):
            ss = P.seqs_of(js)
            ev[js] = np.add.reduceat(b[ss] * V[ss], np.cumsum(P.nact[js]) - P.nact[js])
            np.add.at(V, P.par[js], ev[js])
        if P.J:
            r[1:] += V[1:] - ev[P.seq_inf]
        return V, ev

    @staticmethod
    def post_op(r, variant, t, alpha, beta):
        """the variant's step after ObserveUtility: CFR+ and PCFR+ floor the
        regrets (Alg. 3, Alg. 5); DCFR discounts positive ones by
        t^alpha / (t^alpha + 1), negative ones by t^beta / (t^beta + 1) (Alg. 4)"""
        if variant in (CFR_PLUS, PCFR_PLUS):
            r[1:] = np.maximum(r[1:], 0.0)
        elif variant == DCFR:
            ta, tb = t ** alpha, t ** beta
            fp, fn = ta / (ta + 1.0), tb / (tb + 1.0)
            r[1:] = np.where(r[1:] > 0.0, r[1:] * fp, np.where(r[1:] < 0.0, r[1:] * fn, r[1:]))

    def best_response(self, i, xs):
        """value of player i's best response to the others' sequence-form xs:
        the bottom-up pass of Alg. 1 with ev_j = max_a V[(j, a)] in place of
        the strategy's weighted sum; V[0] is the value"""
        P = self.pl[i]
        V = self.utility(i, xs)
        for js in reversed(P.levels):
            ss = P.seqs_of(js)
            best = np.maximum.reduceat(V[ss], np.cumsum(P.nact[js]) - P.nact[js])
            np.add.at(V, P.par[js], best)
        return float(V[0])


class NOracle:
    """The state of every player and the iteration loop."""

    def __init__(self, tree):
        self.g = NGame(tree)
        self.t = 0
        self.r = [np.zeros(P.S + 1) for P in self.g.pl]
        self.b = [NGame.regret_matching(P, np.zeros(P.S + 1)) for P in self.g.pl]   # uniform
        self.xbar = [np.zeros(P.S + 1) for P in self.g.pl]

    def x(self, i):
        return NGame.sequence_form(self.g.pl[i], self.b[i])

    def _update(self, i, u, xplayed, variant, t, alpha, beta, gamma):
        """player i's half of iteration t: the average (xbar += t^gamma x^t),
        ObserveUtility (Alg. 1), the post-op (Alg. 3-4), NextStrategy; for
        PCFR+ and PCFR, NextStrategy*(m = u) of Alg. 5 (back up r, observe the
        prediction with the previous strategy, regret matching, restore r)"""
        P = self.g.pl[i]
        self.xbar[i] += t ** gamma * xplayed
        NGame.observe_utility(P, u, self.b[i], self.r[i])
        NGame.post_op(self.r[i], variant, t, alpha, beta)
        if variant in (PCFR_PLUS, PCFR):
            rho = self.r[i].copy()
            NGame.observe_utility(P, u, self.b[i], self.r[i])
            self.b[i] = NGame.regret_matching(P, self.r[i])
            self.r[i] = rho
        else:
            self.b[i] = NGame.regret_matching(P, self.r[i])

    def iterate(self, T, variant, alpha=1.5, beta=0.0, gamma=2.0, alternating=True):
        """T iterations; alternating: players 0..n-1 in turn, each seeing the
        strategies the players before it just recomputed (Sec. 3.5.1);
        simultaneous: every utility from the iteration's start"""
        n = self.g.n
        for _ in range(T):
            t = float(self.t + 1)
            xs = [self.x(i) for i in range(n)]
            if alternating:
                for i in range(n):
                    u = self.g.utility(i, xs)
                    self._update(i, u, xs[i], variant, t, alpha, beta, gamma)
                    xs[i] = self.x(i)                 # the players after i see the new x_i
            else:
                us = [self.g.utility(i, xs) for i in range(n)]
                for i in range(n):
                    self._update(i, us[i], xs[i], variant, t, alpha, beta, gamma)
            self.t += 1

    def average_profile(self):
        """xbar_i / xbar_i[0] (the current x_i before any iteration)"""
        return [self.xbar[i] / self.xbar[i][0] if self.xbar[i][0] > 0.0 else self.x(i) for i in range(self.g.n)]

    def nash_conv(self, xs=None):
        """(NashConv, per-player gains) of the profile xs (default: the
        averages): sum over players of best response minus own value, the
        n-player form of the exploitability Sec. 4 reports"""
        xs = self.average_profile() if xs is None else xs
        gains = []
        for i in range(self.g.n):
            v = float(np.dot(xs[i], self.g.utility(i, xs)))
            gains.append(self.g.best_response(i, xs) - v)
        return float(sum(gains)), gains

    def average_strategy(self, i):
        """behavioural average: xbar[(j, a)] / xbar[p_j], uniform where xbar[p_j] = 0"""
        P = self.g.pl[i]
        d = self.xbar[i][P.par[P.seq_inf]]
        return np.where(d > 0.0, self.xbar[i][1:] / np.where(d > 0.0, d, 1.0), 1.0 / P.nact[P.seq_inf])
