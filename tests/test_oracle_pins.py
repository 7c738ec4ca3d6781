"""Pins of the FP64 oracle against things other than itself.

Closed forms (2x2, RPS, fully mixed n x n), the sequence-form LP (von Stengel /
Koller et al., the formulation the paper builds on in Sec. 2.1), brute force
over reduced pure strategies, a tree-walk CFR (same iterates, Sec. 2.1 and
Sec. 5), the paper's Alg. 2 with explicit logic matrices, and invariants
(Ex = e, strategies sum to 1, zero-sum utilities, Zinkevich's regret bound).
"""
import json
import os

import numpy as np
import pytest

from oracle.oracle import Oracle, OracleError
from paper_2605_14277_b300 import games as G
from tests.refimpl import Alg2, ClassicalCFR, SeqForm, brute_force, lp_value

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def tiny_games():
    out = []
    for s in range(6):
        t = G.random_game(100 + s, depth=3, chance={0: 2}, actions=(2, 3), n_classes=2,
                          payoff="int2", name=f"tiny{s}")
        if t.n_nodes <= 30:
            out.append(t)
    for s in range(3):
        t = G.random_game(200 + s, depth=4, chance={1: 2}, actions=(2,), n_classes=2,
                          payoff="int2", name=f"tinyc{s}")
        if t.n_nodes <= 30:
            out.append(t)
    assert len(out) >= 4
    return out


# ---------------------------------------------------------------- closed forms

def test_rps_vanilla_regrets_stay_zero():
    o = Oracle(G.rps())
    o.iterate(50, "cfr")
    for p in (1, 2):
        st = o.get_state(p)
        assert np.all(st["r"] == 0.0)
        assert np.allclose(o.average_strategy(p), 1.0 / 3.0, rtol=0, atol=1e-15)
    e, b1, b2 = o.exploitability()
    assert e == 0.0 and b1 == 0.0 and b2 == 0.0


def test_2x2_golden_closed_form():
    g = json.load(open(os.path.join(GOLD, "matrix2x2.json")))
    o = Oracle(G.matrix_game(g["A"]))
    o.iterate(20000, "cfr+")
    assert np.allclose(o.average_strategy(1), g["p_star"], atol=2e-4)
    assert np.allclose(o.average_strategy(2), g["q_star"], atol=2e-4)
    e, b1, b2 = o.exploitability()
    assert -b2 - 1e-12 <= g["value"] <= b1 + 1e-12
    assert e < 1e-4


@pytest.mark.parametrize("seed", range(5))
def test_2x2_seeded_closed_form(seed):
    A = G.random_2x2_no_saddle(seed)
    a, b, c, d = A.ravel()
    den = a - b - c + d
    p0, q0, v = (d - c) / den, (d - b) / den, (a * d - b * c) / den
    o = Oracle(G.matrix_game(A))
    o.iterate(20000, "cfr+")
    assert abs(o.average_strategy(1)[0] - p0) < 1e-3
    assert abs(o.average_strategy(2)[0] - q0) < 1e-3
    e, b1, b2 = o.exploitability()
    assert -b2 - 1e-12 <= v <= b1 + 1e-12 and e < 1e-3 * (A.max() - A.min())


@pytest.mark.parametrize("n", [3, 4])
def test_fully_mixed_closed_form(n):
    A, p, q, v = G.random_fully_mixed(10 + n, n)
    o = Oracle(G.matrix_game(A))
    o.iterate(20000, "cfr+")
    assert np.allclose(o.average_strategy(1), p, atol=2e-3)
    assert np.allclose(o.average_strategy(2), q, atol=2e-3)
    e, b1, b2 = o.exploitability()
    assert -b2 - 1e-12 <= v <= b1 + 1e-12


# ------------------------------------------------------------------ LP / brute force

def test_brute_force_equals_sequence_form_lp():
    for t in tiny_games():
        sf = SeqForm(t)
        v, _, _ = lp_value(sf)
        vb, nx, ny = brute_force(sf)
        assert abs(v - vb) < 1e-9, t.name


@pytest.mark.parametrize("variant", ["cfr", "cfr+", "dcfr", "pcfr+", "pcfr"])
def test_oracle_brackets_lp_value(variant):
    games = tiny_games() + [G.small_random_game(1)]
    for t in games:
        sf = SeqForm(t)
        v, x, y = lp_value(sf)
        o = Oracle(t)
        o.iterate(3000, variant)
        e, b1, b2 = o.exploitability()
        assert -b2 - 1e-9 <= v <= b1 + 1e-9, (t.name, v, b1, b2)
        assert e <= 0.01 * t.payoff_range(), (t.name, e)


def test_lp_equilibrium_has_zero_exploitability():
    for t in tiny_games() + [G.small_random_game(1)]:
        sf = SeqForm(t)
        v, x, y = lp_value(sf)
        o = Oracle(t)
        e, b1, b2 = o.exploitability_of(x, y)
        assert abs(e) < 1e-8 and abs(b1 - v) < 1e-8 and abs(-b2 - v) < 1e-8, t.name


def test_poker_value_against_lp():
    t = G.poker_game()
    sf = SeqForm(t)
    v, x, y = lp_value(sf)
    o = Oracle(t)
    e, b1, b2 = o.exploitability_of(x, y)
    assert abs(e) < 1e-7
    o.iterate(2000, "dcfr")
    e, b1, b2 = o.exploitability()
    assert -b2 - 1e-9 <= v <= b1 + 1e-9
    assert e < 1e-3


def test_poker_node_count_matches_table1():
    g = json.load(open(os.path.join(GOLD, "poker_counts.json")))
    t = G.poker_game()
    assert g["lo"] <= t.n_nodes < g["hi"]


# ------------------------------------------------------------------ equivalences

def test_payoff_matrix_products():
    for t in [G.small_random_game(1), G.poker_game()]:
        sf = SeqForm(t)
        o = Oracle(t)
        rng = np.random.default_rng(0)
        x = rng.uniform(size=sf.S[1] + 1)
        y = rng.uniform(size=sf.S[2] + 1)
        assert np.allclose(o.utility(1, y), sf.M @ y, rtol=1e-13, atol=1e-13)
        assert np.allclose(o.utility(2, x), -(sf.M.T @ x), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("variant,alt,gamma", [("cfr", False, 0.0), ("cfr+", True, 1.0),
                                               ("dcfr", True, 2.0), ("pcfr+", True, 2.0),
                                               ("cfr+", False, 1.0), ("dcfr", False, 2.0),
                                               ("pcfr", True, 0.0), ("pcfr", False, 1.0)])
def test_classical_cfr_same_iterates(variant, alt, gamma):
    # continuous payoffs: with integer payoffs, mathematically-zero regrets come
    # out as +-1e-17 in one formulation and 0 in the other, and regret matching's
    # zero test sends the iterates apart (the divergence noted in Appendix D)
    cont = G.random_game(1, depth=6, chance={0: 3}, actions=(2, 3), payoff="normal")
    for t in [cont, G.poker_game()]:
        n_it = 12 if t.n_nodes > 1000 else 40
        sf = SeqForm(t)
        o = Oracle(t)
        o.iterate(n_it, variant, alternating=alt, gamma=gamma)
        c = ClassicalCFR(t)
        c.iterate(n_it, variant, alternating=alt, alpha=1.5, beta=0.0, gamma=gamma)
        for p in (1, 2):
            r_o = o.get_state(p)["r"]
            r_c = c.regrets(p, sf)
            assert np.allclose(r_o, r_c, rtol=1e-10, atol=1e-10 * max(1.0, np.abs(r_c).max()))
            assert np.allclose(o.average_strategy(p), c.average(p, sf), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("alt", [True, False])
def test_classical_cfr_same_iterates_dcfr_other_parameters(alt):
    # DCFR with beta != 0 (the negative-regret factor t^b/(t^b+1) then varies
    # with t) and a cubic average, against the tree walk
    t = G.random_game(2, depth=6, chance={0: 3}, actions=(2, 3), payoff="normal")
    sf = SeqForm(t)
    o = Oracle(t)
    o.iterate(30, "dcfr", alpha=1.0, beta=0.5, gamma=3.0, alternating=alt)
    c = ClassicalCFR(t)
    c.iterate(30, "dcfr", alternating=alt, alpha=1.0, beta=0.5, gamma=3.0)
    for p in (1, 2):
        r_c = c.regrets(p, sf)
        assert np.allclose(o.get_state(p)["r"], r_c, rtol=1e-10, atol=1e-10 * max(1.0, np.abs(r_c).max()))
        assert np.allclose(o.average_strategy(p), c.average(p, sf), rtol=1e-10, atol=1e-12)


def test_alg2_literal_matches_oracle_steps():
    rng = np.random.default_rng(3)
    for t in [G.small_random_game(1), G.poker_game()] + tiny_games()[:2]:
        sf = SeqForm(t)
        o = Oracle(t)
        for p in (1, 2):
            A2 = Alg2(sf, p)
            r = rng.standard_normal(sf.S[p])
            r[rng.uniform(size=r.shape) < 0.3] = -1.0  # some infosets with all-negative regrets
            b2, x2 = A2.next_strategy(r)
            b_o = o.regret_matching(p, r)
            x_o = o.sequence_form(p, b_o)
            assert np.allclose(b_o, b2, rtol=1e-14, atol=1e-15)
            assert np.allclose(x_o, x2, rtol=1e-14, atol=1e-15)
            u = rng.standard_normal(sf.S[p] + 1)
            r_o, V, ev = o.observe_utility(p, u, b_o, r)
            r_2, q = A2.observe_utility(u, b2, r)
            assert np.allclose(r_o, r_2, rtol=1e-12, atol=1e-12)
            assert np.allclose(V[1:], q, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ invariants

def test_sequence_form_constraints_and_simplex():
    t = G.poker_game()
    sf = SeqForm(t)
    o = Oracle(t)
    o.iterate(37, "dcfr")
    for p in (1, 2):
        E, e = sf.constraints(p)
        st = o.get_state(p)
        b = st["b"]
        na = sf.nact[p]
        sums = np.add.reduceat(b, sf.off[p])
        assert np.allclose(sums, 1.0, atol=1e-14)
        x = o.sequence_form(p, b)
        assert np.abs(E @ x - e).max() < 1e-12
        xb = st["xbar"] / st["xbar"][0]
        assert np.abs(E @ xb - e).max() < 1e-12
        assert (b >= 0).all() and (x >= 0).all()


def test_zero_sum_utilities():
    t = G.small_random_game(1)
    o = Oracle(t)
    rng = np.random.default_rng(1)
    for _ in range(5):
        b1 = o.regret_matching(1, rng.standard_normal(o.S[1]))
        b2 = o.regret_matching(2, rng.standard_normal(o.S[2]))
        x, y = o.sequence_form(1, b1), o.sequence_form(2, b2)
        v1 = x @ o.utility(1, y)
        v2 = y @ o.utility(2, x)
        assert abs(v1 + v2) < 1e-12


def test_cfr_plus_regrets_nonnegative():
    o = Oracle(G.poker_game())
    o.iterate(25, "cfr+")
    for p in (1, 2):
        assert (o.get_state(p)["r"] >= 0).all()


@pytest.mark.parametrize("T", [10, 100, 1000])
def test_regret_bound(T):
    """Vanilla simultaneous CFR, uniform averaging: T * (BR1 + BR2) = R1 + R2
    and R_i <= sum_j max_a (r_j[a])^+ <= Delta J_i sqrt(max|A|) sqrt(T)
    (Zinkevich et al. 2007, Thm. 3-4)."""
    t = G.small_random_game(1)
    sf = SeqForm(t)
    o = Oracle(t)
    o.iterate(T, "cfr")
    e, b1, b2 = o.exploitability()
    gap_T = 2.0 * e * T
    pos = 0.0
    for p in (1, 2):
        r = o.get_state(p)["r"]
        pos += sum(max(0.0, r[sf.off[p][j]: sf.off[p][j] + sf.nact[p][j]].max())
                   for j in range(len(sf.nact[p])))
    assert gap_T <= pos + 1e-9
    delta = t.payoff_range()
    bound = sum(delta * len(sf.nact[p]) * np.sqrt(sf.nact[p].max()) * np.sqrt(T) for p in (1, 2))
    assert pos <= bound


# ------------------------------------------------------------------ validation

def _copy(t):
    return G.Tree(t.parent.copy(), t.kind.copy(), t.infoset.copy(), t.action.copy(),
                  t.chance_prob.copy(), t.payoff.copy())


def test_rejects_malformed_trees():
    base = G.small_random_game(1)
    Oracle(base)
    # imperfect recall: merge two player-1 infosets with different own histories
    t = _copy(base)
    p1 = np.nonzero(t.kind == 1)[0]
    deep = [i for i in p1 if t.infoset[i] != t.infoset[p1[0]] and t.infoset[i] > 5]
    same_na = [i for i in deep if (t.parent == i).sum() == (t.parent == p1[0]).sum()]
    t.infoset[same_na[-1]] = t.infoset[p1[0]]
    with pytest.raises(OracleError):
        Oracle(t)
    # chance probabilities that do not sum to one
    t = _copy(base)
    t.chance_prob[1] = 0.5
    with pytest.raises(OracleError):
        Oracle(t)
    # NaN payoff
    t = _copy(base)
    t.payoff[-1] = np.nan
    with pytest.raises(OracleError):
        Oracle(t)
    # duplicated action label
    t = _copy(base)
    kids = np.nonzero(t.parent == 0)[0]
    t.action[kids[1]] = t.action[kids[0]]
    with pytest.raises(OracleError):
        Oracle(t)
