"""Host game compiler: every validity rule rejects its own kind of invalid tree
with its own message, and valid trees (including ones with chance nodes at
several depths and a terminal root) compile.  CPU only (the layout probe
calls the compiler directly)."""
import numpy as np
import pytest

from paper_2605_14277_b300 import games as G
from tests.layout_probe import Layout


def copy(t):
    return G.Tree(t.parent.copy(), t.kind.copy(), t.infoset.copy(), t.action.copy(), t.chance_prob.copy(),
                  t.payoff.copy())


def small():
    return G.small_random_game(1)   # root chance node (3 outcomes), both players, integer payoffs


def first(t, pred):
    return int(np.nonzero(pred)[0][0])


def bad_kind(t):
    t.kind[first(t, t.kind == 3)] = 7


def parent_after_child(t):
    i = first(t, np.arange(t.n_nodes) > 2)
    t.parent[i] = i


def terminal_with_children(t):
    i = first(t, t.kind == 3)
    j = first(t, (np.arange(t.n_nodes) > i))
    t.parent[j] = i


def decision_without_infoset(t):
    t.infoset[first(t, t.kind == 1)] = -1


def non_finite_payoff(t):
    t.payoff[first(t, t.kind == 3)] = np.nan


def nonterminal_without_children(t):
    # the last node made a decision node: nothing can follow it
    t.kind[-1] = 1
    t.infoset[-1] = t.infoset[t.kind == 1].max() + 1


def action_out_of_range(t):
    i = first(t, (t.parent >= 0) & (t.kind[np.maximum(t.parent, 0)] == 1))
    t.action[i] = 99


def duplicate_action(t):
    # two children of one decision node get the same label
    p = t.parent
    for i in range(1, t.n_nodes):
        sib = np.nonzero(p == p[i])[0]
        if t.kind[p[i]] == 1 and len(sib) >= 2:
            t.action[sib[1]] = t.action[sib[0]]
            return
    raise AssertionError("no decision node with two children")


def bad_probability(t):
    t.chance_prob[first(t, (t.parent >= 0) & (t.kind[np.maximum(t.parent, 0)] == 0))] = 1.5


def probabilities_not_one(t):
    t.chance_prob[first(t, (t.parent >= 0) & (t.kind[np.maximum(t.parent, 0)] == 0))] *= 0.5


def action_count_mismatch(t):
    # a node of a two-node infoset moves to an infoset with another action count
    d = np.nonzero(t.kind == 1)[0]
    na = {int(t.infoset[i]): int((t.parent == i).sum()) for i in d}
    for i in d:
        for j, a in na.items():
            if a != na[int(t.infoset[i])]:
                t.infoset[i] = j
                return
    raise AssertionError("every infoset has the same action count")


def ids_not_dense(t):
    t.infoset[first(t, t.kind == 1)] = t.infoset[t.kind == 1].max() + 5


def imperfect_recall(t):
    # two player-1 nodes with different own histories share an infoset
    d = np.nonzero(t.kind == 1)[0]
    deep = [i for i in d if t.parent[i] >= 0 and any(t.kind[a] == 1 for a in ancestors(t, i))]
    shallow = [i for i in d if not any(t.kind[a] == 1 for a in ancestors(t, i))]
    i, j = deep[0], shallow[0]
    if (t.parent == i).sum() == (t.parent == j).sum():
        t.infoset[i] = t.infoset[j]
        return
    for j in shallow:
        if (t.parent == i).sum() == (t.parent == j).sum():
            t.infoset[i] = t.infoset[j]
            return
    raise AssertionError("no pair with equal action counts")


def ancestors(t, i):
    out = []
    while t.parent[i] >= 0:
        i = t.parent[i]
        out.append(i)
    return out


CASES = [
    (bad_kind, "bad node kind"),
    (parent_after_child, "parent must precede child"),
    (terminal_with_children, "terminal with children"),
    (decision_without_infoset, "decision node without infoset"),
    (non_finite_payoff, "non-finite payoff"),
    (nonterminal_without_children, "non-terminal without children"),
    (action_out_of_range, "action label out of range"),
    (duplicate_action, "duplicate action label"),
    (bad_probability, "bad chance probability"),
    (probabilities_not_one, "do not sum to 1"),
    (action_count_mismatch, "action-count mismatch"),
    (ids_not_dense, "not dense"),
    (imperfect_recall, "imperfect recall"),
]


@pytest.mark.parametrize("spoil,msg", CASES, ids=[c[1] for c in CASES])
def test_invalid_tree_rejected(spoil, msg):
    t = copy(small())
    spoil(t)
    with pytest.raises(ValueError, match=msg):
        Layout([t])
    # and inside a batch: the message names the game
    with pytest.raises(ValueError, match="game 1: .*" + msg):
        Layout([small(), t])


def test_valid_trees_compile():
    for t in (small(), G.poker_game(), G.rps(),
              G.random_game(5, depth=5, chance={0: 3, 3: 2}, actions=(2, 3), payoff="normal")):
        Layout([t])
    # a terminal root: no decision for either player
    root = G.Tree(np.array([-1], np.int32), np.array([3], np.int8), np.array([-1], np.int32),
                  np.array([0], np.int32), np.array([1.0]), np.array([2.5]))
    lay = Layout([root])
    assert lay.pl[0]["inf_seq"].tolist() == [0, 1] and lay.pl[1]["inf_seq"].tolist() == [0, 1]
