"""Pins of the n-player FP64 oracle (oracle/nplayer.py) to things other than itself.

* The two-player reduction: on a two-player game, written as an n-player game
  with n = 2 or with a third player who never acts (payoff 0), every iterate
  equals the two-player C oracle's (oracle/cfr_oracle.c, itself pinned in
  test_oracle_pins.py), for every variant and both schedules, and NashConv is
  twice its exploitability (BR1 + BR2) / 2.
* Utilities by a tree walk: u_i[s] re-derived from the game tree with
  behavioural probabilities multiplied down each path (no sequence form).
* Best responses by brute force over every pure strategy of the player.
* Zero-sum games: the players' values sum to 0.
* A dense normal-form game: the payoff tensors contracted with einsum, and one
  alternating CFR iteration written out from Alg. 1 by hand.
"""
import itertools

import numpy as np
import pytest

from paper_2605_14277_b300 import games as G
from oracle.nplayer import CFR, CFR_PLUS, DCFR, NGame, NOracle, PCFR, PCFR_PLUS

VARIANTS = {"cfr": (CFR, (0.0, 0.0, 0.0)), "cfr+": (CFR_PLUS, (0.0, 0.0, 1.0)), "dcfr": (DCFR, (1.5, 0.0, 2.0)),
            "pcfr+": (PCFR_PLUS, (0.0, 0.0, 2.0)), "pcfr": (PCFR, (0.0, 0.0, 0.0))}


def rel_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max())) if a.size else 0.0


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("alternating", [True, False])
def test_two_player_reduction(variant, alternating):
    from oracle.oracle import Oracle
    v, (a, b, g) = VARIANTS[variant]
    for tree in (G.small_random_game(1), G.small_random_game(2), G.poker_game()):
        o = Oracle(tree)
        o.iterate(40, variant, a, b, g, alternating=alternating)
        e, _, _ = o.exploitability()
        for n in (2, 3):
            no = NOracle(G.nplayer_from_two_player(tree, n))
            no.iterate(40, v, a, b, g, alternating=alternating)
            for p in (1, 2):
                st = o.get_state(p)
                assert rel_err(no.r[p - 1][1:], st["r"]) < 1e-9
                assert rel_err(no.b[p - 1][1:], st["b"]) < 1e-9
                assert rel_err(no.xbar[p - 1], st["xbar"]) < 1e-9
            nc, gains = no.nash_conv()
            assert nc == pytest.approx(2 * e, rel=1e-9, abs=1e-12)
            if n == 3:
                assert gains[2] == pytest.approx(0.0, abs=1e-12)   # a player who never acts gains nothing


def random_behaviour(game: NGame, rng):
    out = []
    for P in game.pl:
        b = np.zeros(P.S + 1)
        for j in range(P.J):
            w = rng.random(P.nact[j]) + 0.05
            b[P.off[j]:P.off[j] + P.nact[j]] = w / w.sum()
        out.append(b)
    return out


def tree_walk_utilities(tree, bs):
    """u_i by walking the tree: the reach of every player's behaviour and of
    chance, multiplied down each path; u_i[own last sequence at z] +=
    pi_c(z) prod_{k != i} pi_k(z) payoff_i(z)."""
    n = tree.n_players
    N = tree.n_nodes
    # caller sequence numbering: 1 + actions of the infosets before j + a
    nact = [dict() for _ in range(n)]
    for i in range(1, N):
        q = tree.parent[i]
        if tree.kind[q] == G.N_DECISION:
            key = int(tree.infoset[q])
            nact[tree.actor[q]][key] = max(nact[tree.actor[q]].get(key, 0), int(tree.action[i]) + 1)
    off = []
    for p in range(n):
        o, s = {}, 1
        for j in sorted(nact[p]):
            o[j] = s
            s += nact[p][j]
        off.append(o)
    reach = np.ones((N, n + 1))          # [..., n] is chance
    own = np.zeros((N, n), np.int64)
    for i in range(1, N):
        q = tree.parent[i]
        reach[i] = reach[q]
        own[i] = own[q]
        if tree.kind[q] == G.N_CHANCE:
            reach[i, n] *= tree.chance_prob[i]
        elif tree.kind[q] == G.N_DECISION:
            p = tree.actor[q]
            s = off[p][int(tree.infoset[q])] + int(tree.action[i])
            reach[i, p] *= bs[p][s]
            own[i, p] = s
    us = [np.zeros(len(b)) for b in bs]
    for z in np.flatnonzero(tree.kind == G.N_TERMINAL):
        for i in range(n):
            others = np.prod([reach[z, k] for k in range(n) if k != i])
            us[i][own[z, i]] += reach[z, n] * others * tree.payoff[z, i]
    return us


NGAMES = [lambda: G.kuhn3_game(), lambda: G.small_nplayer_game(3, 1), lambda: G.small_nplayer_game(3, 2),
          lambda: G.random_nplayer_game(4, 7, depth=8, chance={0: 3, 4: 2}, actions=(2, 3)),
          lambda: G.random_nplayer_game(5, 3, depth=6, chance={0: 2}, actions=(2, 3), zero_sum=False)]


@pytest.mark.parametrize("k", range(len(NGAMES)))
def test_utilities_match_tree_walk(k):
    tree = NGAMES[k]()
    game = NGame(tree)
    rng = np.random.default_rng(k)
    bs = random_behaviour(game, rng)
    xs = [NGame.sequence_form(P, b) for P, b in zip(game.pl, bs)]
    # the sequence-form constraints: sum_a x[(j,a)] = x[p_j]
    for P, x in zip(game.pl, xs):
        assert x[0] == 1.0
        for j in range(P.J):
            assert x[P.off[j]:P.off[j] + P.nact[j]].sum() == pytest.approx(x[P.par[j]], rel=1e-12, abs=1e-15)
    walk = tree_walk_utilities(tree, bs)
    for i in range(tree.n_players):
        assert rel_err(game.utility(i, xs), walk[i]) < 1e-12


@pytest.mark.parametrize("k", range(len(NGAMES) - 1))
def test_zero_sum_values_sum_to_zero(k):
    tree = NGAMES[k]()
    game = NGame(tree)
    bs = random_behaviour(game, np.random.default_rng(10 + k))
    xs = [NGame.sequence_form(P, b) for P, b in zip(game.pl, bs)]
    vals = [float(np.dot(xs[i], game.utility(i, xs))) for i in range(tree.n_players)]
    assert abs(sum(vals)) < 1e-12 * max(1.0, max(abs(v) for v in vals))


def test_best_response_by_brute_force():
    rng = np.random.default_rng(5)
    for seed in range(4):
        tree = G.random_nplayer_game(3, 100 + seed, depth=4, chance={0: 2}, actions=(2,), n_classes=2)
        game = NGame(tree)
        bs = random_behaviour(game, rng)
        xs = [NGame.sequence_form(P, b) for P, b in zip(game.pl, bs)]
        for i in range(3):
            P = game.pl[i]
            assert P.J <= 10
            best = -np.inf
            for choice in itertools.product(*[range(P.nact[j]) for j in range(P.J)]):
                pure = np.zeros(P.S + 1)
                for j, a in enumerate(choice):
                    pure[P.off[j] + a] = 1.0
                b2 = list(bs)
                b2[i] = pure
                walk = tree_walk_utilities(tree, b2)
                # the pure strategy's value: sum over its own reach-1 sequences
                xp = NGame.sequence_form(P, pure)
                best = max(best, float(np.dot(xp, walk[i])))
            assert game.best_response(i, xs) == pytest.approx(best, rel=1e-12, abs=1e-12)


def test_normal_form_tensors_and_one_iteration_by_hand():
    rng = np.random.default_rng(3)
    A = [rng.standard_normal((2, 3, 2)) for _ in range(3)]
    tree = G.nplayer_normal_form(A)
    game = NGame(tree)
    # utilities = the dense tensors contracted with einsum
    xs = [np.concatenate([[1.0], rng.dirichlet(np.ones(k))]) for k in (2, 3, 2)]
    y = [x[1:] for x in xs]
    want = [np.einsum("abc,b,c->a", A[0], y[1], y[2]), np.einsum("abc,a,c->b", A[1], y[0], y[2]),
            np.einsum("abc,a,b->c", A[2], y[0], y[1])]
    for i in range(3):
        assert rel_err(game.utility(i, xs)[1:], want[i]) < 1e-13
    # one alternating vanilla CFR iteration from uniform strategies (Alg. 1):
    # r_i = u_i - <b_i, u_i>, b_i' = RM(r_i), later players see b_i'
    def rm(r):
        q = np.maximum(r, 0.0)
        return q / q.sum() if q.sum() > 0 else np.full(len(r), 1.0 / len(r))
    b = [np.full(2, 0.5), np.full(3, 1 / 3), np.full(2, 0.5)]
    rs = []
    u0 = np.einsum("abc,b,c->a", A[0], b[1], b[2])
    rs.append(u0 - b[0] @ u0)
    b[0] = rm(rs[0])
    u1 = np.einsum("abc,a,c->b", A[1], b[0], b[2])
    rs.append(u1 - b[1] @ u1)
    b[1] = rm(rs[1])
    u2 = np.einsum("abc,a,b->c", A[2], b[0], b[1])
    rs.append(u2 - b[2] @ u2)
    b[2] = rm(rs[2])
    o = NOracle(tree)
    o.iterate(1, CFR, 0.0, 0.0, 0.0, alternating=True)
    for i in range(3):
        assert rel_err(o.r[i][1:], rs[i]) < 1e-13
        assert rel_err(o.b[i][1:], b[i]) < 1e-13
        assert rel_err(o.xbar[i][1:], np.full(len(b[i]), 1.0 / len(b[i]))) < 1e-15   # t^0 * uniform


def test_dummy_player_changes_nothing_for_three_players():
    """A fourth player who never acts leaves a 3-player game's iterates unchanged."""
    base = G.small_nplayer_game(3, 2)
    pay = np.zeros((base.n_nodes, 4))
    pay[:, :3] = base.payoff
    four = G.NTree(4, base.parent, base.kind, base.actor, base.infoset, base.action, base.chance_prob, pay)
    o3, o4 = NOracle(base), NOracle(four)
    o3.iterate(30, DCFR, 1.5, 0.0, 2.0)
    o4.iterate(30, DCFR, 1.5, 0.0, 2.0)
    for i in range(3):
        assert np.array_equal(o3.r[i], o4.r[i]) and np.array_equal(o3.xbar[i], o4.xbar[i])
