"""CUDA path (libcfr.so through its C ABI) against the FP64 oracle.

Tolerances: one iteration from identical state, norm-wise relative error
<= 1e-5 per vector; exploitability of identical strategies (FP64 on both
sides) <= 1e-9.  Trajectories: independent runs of correct implementations
drift apart (regret matching's sensitivity, Appendix D); the oracle itself
differs from a summation-order variant of itself by 7-38% in final
exploitability after 10^4 iterations.  So along a trajectory every checkpoint
is re-synchronised (one iteration from the GPU's own state must match the
oracle), and the final exploitability must lie inside the spread of FP64
oracle runs that differ only below the level of any meaningful change.
"""
import zlib

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2605_14277_b300 import games as G
from tests.parity_util import EXPL_RTOL, ONE_STEP_RTOL, random_state, rel, strategy_mismatch_ok

pytestmark = pytest.mark.gpu

VARIANTS = ["cfr", "cfr+", "dcfr", "pcfr+", "pcfr"]


@pytest.fixture(scope="module")
def cfr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_14277_b300 import cfr as C
    return C


def parity_games():
    return {
        "small_int": G.small_random_game(1),
        "small_normal": G.random_game(1, depth=6, chance={0: 3}, actions=(2, 3), payoff="normal"),
        "poker": G.poker_game(),
        "two_chance": G.random_game(11, depth=8, chance={0: 4, 4: 3}, actions=(2, 3, 4), payoff="normal"),
        "rps": G.rps(),
        "mixed3": G.matrix_game(G.random_fully_mixed(3, 3)[0]),
    }


def one_step(cfr, tree, variant, mode, seed, game_in_batch=None, **load):
    o = Oracle(tree)
    rng = np.random.default_rng(seed)
    if game_in_batch is None:
        s = cfr.Solver(tree, **load)
        gi = 0
    else:
        others, gi = game_in_batch
        trees = list(others)
        trees.insert(gi, tree)
        s = cfr.Solver(trees, **load)
    s.set_update_mode(mode)
    for p in (1, 2):
        r, b, xb, t = random_state(o, p, rng)
        o.set_state(p, r, b, xb, t)
        s.set_state(p, r, b, xb, t, game=gi)
    alt = {"alternating": True, "simultaneous": False}[mode]
    o.iterate(1, variant, alternating=alt)
    s.iterate(1, variant)
    out = {p: (s.get_state(p, game=gi), o.get_state(p)) for p in (1, 2)}
    return o, s, out


@pytest.mark.parametrize("name", list(parity_games()))
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("mode", ["alternating", "simultaneous"])
def test_one_iteration_from_identical_state(cfr, name, variant, mode):
    tree = parity_games()[name]
    o, s, out = one_step(cfr, tree, variant, mode, seed=zlib.crc32(f"{name}/{variant}/{mode}".encode()))
    for p in (1, 2):
        g_, o_ = out[p]
        assert g_["t"] == o_["t"] == 6
        assert rel(g_["r"], o_["r"]) <= ONE_STEP_RTOL, ("r", p)
        assert rel(g_["xbar"], o_["xbar"]) <= ONE_STEP_RTOL, ("xbar", p)
        _, na = o.infosets(p)
        assert strategy_mismatch_ok(g_["b"], o_["b"], o_["r"], na) == 0, ("b", p)


@pytest.mark.parametrize("variant,alpha,beta,gamma", [("dcfr", 1.0, 0.5, 3.0), ("dcfr", 2.0, -0.5, 0.0),
                                                      ("pcfr", 0.0, 0.0, 1.5), ("cfr+", 0.0, 0.0, 2.0)])
@pytest.mark.parametrize("mode", ["alternating", "simultaneous"])
def test_one_iteration_other_parameters(cfr, variant, alpha, beta, gamma, mode):
    # non-default discount and averaging exponents (the per-iteration
    # parameter table), one iteration from identical state
    tree = G.random_game(11, depth=8, chance={0: 4, 4: 3}, actions=(2, 3, 4), payoff="normal")
    o = Oracle(tree)
    s = cfr.Solver(tree)
    s.set_update_mode(mode)
    rng = np.random.default_rng(zlib.crc32(f"{variant}/{alpha}/{beta}/{gamma}/{mode}".encode()))
    for p in (1, 2):
        r, b, xb, t = random_state(o, p, rng)
        o.set_state(p, r, b, xb, t)
        s.set_state(p, r, b, xb, t)
    o.iterate(1, variant, alpha=alpha, beta=beta, gamma=gamma, alternating=(mode == "alternating"))
    s.iterate(1, variant, alpha=alpha, beta=beta, gamma=gamma)
    for p in (1, 2):
        g_, o_ = s.get_state(p), o.get_state(p)
        assert rel(g_["r"], o_["r"]) <= ONE_STEP_RTOL, ("r", p)
        assert rel(g_["xbar"], o_["xbar"]) <= ONE_STEP_RTOL, ("xbar", p)
        _, na = o.infosets(p)
        assert strategy_mismatch_ok(g_["b"], o_["b"], o_["r"], na) == 0, ("b", p)


def test_one_iteration_inside_a_batch(cfr):
    others = [G.sized_random_game(40 + k, 10 ** (2 + k % 3)) for k in range(5)]
    tree = G.poker_game()
    for variant in VARIANTS:
        o, s, out = one_step(cfr, tree, variant, "alternating", seed=3, game_in_batch=(others, 2))
        for p in (1, 2):
            g_, o_ = out[p]
            assert rel(g_["r"], o_["r"]) <= ONE_STEP_RTOL
            assert rel(g_["xbar"], o_["xbar"]) <= ONE_STEP_RTOL


@pytest.mark.parametrize("passes", [1, 2])
def test_every_launch_choice_matches_oracle(cfr, passes):
    """Every launch shape x unit layout, with each player's two passes fused
    into one launch or split into two: one iteration from identical state
    matches the oracle, for a game alone and inside a batch."""
    tree = parity_games()["two_chance"]
    others = [G.sized_random_game(60 + k, 10 ** (2 + k % 3)) for k in range(3)]
    for shape in range(1, cfr.lib().cfr_num_shapes() + 1):
        for flat in (False, True):
            for gib in (None, (others, 1)):
                o, s, out = one_step(cfr, tree, "dcfr", "alternating", seed=shape, game_in_batch=gib,
                                     shape=shape, flat=flat, passes=passes)
                for p in (1, 2):
                    g_, o_ = out[p]
                    assert rel(g_["r"], o_["r"]) <= ONE_STEP_RTOL, (shape, flat, p)
                    assert rel(g_["xbar"], o_["xbar"]) <= ONE_STEP_RTOL, (shape, flat, p)
                s.close()


def test_fused_and_split_passes_are_identical(cfr):
    """The fused half-step (one launch per player) and the split passes run
    the same arithmetic on the same units: bit-identical state after many
    launches, with games masked off part of the time."""
    trees = [G.sized_random_game(3000 + k, 10 ** (2 + k % 4)) for k in range(6)] + [G.poker_game()]
    a = cfr.Solver(trees, passes=1)
    b = cfr.Solver(trees, passes=2)
    mask = [1, 0, 1, 1, 0, 1, 1]
    for s in (a, b):
        s.iterate(70, "pcfr+")
        s.iterate(65, "pcfr+", active=mask)
        s.iterate(130, "dcfr")
    for g in range(len(trees)):
        for p in (1, 2):
            x, y = a.get_state(p, game=g), b.get_state(p, game=g)
            assert x["t"] == y["t"]
            for k in ("r", "b", "xbar"):
                assert np.array_equal(x[k], y[k]), (g, p, k)


def test_exploitability_fp64_matches_oracle(cfr):
    for tree in [G.poker_game(), G.small_random_game(1),
                 G.random_game(11, depth=8, chance={0: 4, 4: 3}, actions=(2, 3, 4), payoff="normal")]:
        o = Oracle(tree)
        o.iterate(37, "dcfr")
        s = cfr.Solver(tree)
        for p in (1, 2):
            st = o.get_state(p)
            s.set_state(p, st["r"], st["b"], st["xbar"], st["t"])
        e_o, b1_o, b2_o = o.exploitability()
        e_g, b1_g, b2_g = s.exploitability()
        assert abs(b1_g - b1_o) <= 1e-10 * max(1.0, abs(b1_o))
        assert abs(b2_g - b2_o) <= 1e-10 * max(1.0, abs(b2_o))
        assert abs(e_g - e_o) <= 1e-9 * max(abs(e_o), 1e-12)


def test_average_strategy_matches_oracle(cfr):
    """behavioural average of the same state, computed by both sides (FP64)"""
    tree = G.poker_game()
    s = cfr.Solver(tree)
    s.iterate(200, "cfr+")
    o = Oracle(tree)
    for p in (1, 2):
        st = s.get_state(p)
        o.set_state(p, st["r"], st["b"], st["xbar"], st["t"])
    for p in (1, 2):
        assert np.abs(s.average_strategy(p) - o.average_strategy(p)).max() < 1e-12


def test_rps_vanilla_stays_uniform(cfr):
    s = cfr.Solver(G.rps())
    s.iterate(100, "cfr")
    for p in (1, 2):
        st = s.get_state(p)
        assert np.all(st["r"] == 0.0)
        assert np.allclose(s.average_strategy(p), 1 / 3, atol=1e-7)
    assert abs(s.exploitability()[0]) < 1e-7


def relabel(t, seed):
    """Same game, infoset ids permuted: only the oracle's summation order changes."""
    rng = np.random.default_rng(seed)
    inf = t.infoset.copy()
    for p in (1, 2):
        m = t.kind == p
        inf[m] = rng.permutation(inf[m].max() + 1)[inf[m]]
    return G.Tree(t.parent, t.kind, inf, t.action, t.chance_prob, t.payoff)


def perturb(t, seed, eps=1e-12):
    """Same game up to payoffs scaled by 1 + 1e-12 N(0,1): exploitability moves
    by at most ~1e-12 of the payoff scale, rounding in the iterates changes."""
    rng = np.random.default_rng(seed)
    return G.Tree(t.parent, t.kind, t.infoset, t.action, t.chance_prob,
                  t.payoff * (1.0 + eps * rng.standard_normal(t.payoff.shape)))


def oracle_spread(tree, variant, T):
    """Final exploitability of FP64 oracle runs that differ from the game only
    at the level of the GPU's arithmetic: the game itself, two relabellings of
    its infosets (summation order), three 1e-12 payoff perturbations and three
    at FP32 rounding level (1e-7; the passes run in FP32)."""
    games = [tree, relabel(tree, 1), relabel(tree, 2), perturb(tree, 1), perturb(tree, 2), perturb(tree, 3),
             perturb(tree, 4, 1e-7), perturb(tree, 5, 1e-7), perturb(tree, 6, 1e-7)]
    runs = []
    for t in games:
        o = Oracle(t)
        o.iterate(T, variant)
        runs.append(o.exploitability()[0])
    lo, hi = min(runs), max(runs)
    return lo, hi, max(hi / lo, 1.0 + EXPL_RTOL), runs


def check_step_from_gpu_state(s, tree, variant):
    """One more iteration from the GPU's own (late) state on both sides."""
    o = Oracle(tree)
    for p in (1, 2):
        st = s.get_state(p)
        o.set_state(p, st["r"], st["b"], st["xbar"], st["t"])
    # exploitability of exactly these averages: FP64 on both sides
    e_o, b1_o, b2_o = o.exploitability()
    e_g, b1_g, b2_g = s.exploitability()
    assert abs(b1_g - b1_o) <= 1e-9 * max(1.0, abs(b1_o)) and abs(b2_g - b2_o) <= 1e-9 * max(1.0, abs(b2_o))
    o.iterate(1, variant)
    s.iterate(1, variant)
    for p in (1, 2):
        g_, o_ = s.get_state(p), o.get_state(p)
        assert rel(g_["r"], o_["r"]) <= ONE_STEP_RTOL
        assert rel(g_["xbar"], o_["xbar"]) <= ONE_STEP_RTOL
        _, na = o.infosets(p)
        assert strategy_mismatch_ok(g_["b"], o_["b"], o_["r"], na) == 0
    return e_g


@pytest.mark.parametrize("variant", ["cfr+", "dcfr", "pcfr+", "pcfr"])
def test_poker_trajectory_10k(cfr, variant):
    """Poker, 10^4 iterations: one iteration from the GPU's state at t = 1000,
    5000 and 9999 matches the oracle (1e-5) and both compute the same FP64
    exploitability of its averages (1e-9); the final exploitability lies in
    the oracle's own spread."""
    tree = G.poker_game()
    s = cfr.Solver(tree)
    done = 0
    for t in (1000, 5000, 9999):
        s.iterate(t - done, variant)
        check_step_from_gpu_state(s, tree, variant)
        done = t + 1
    s.iterate(10000 - done, variant)
    e_g = s.exploitability()[0]
    lo, hi, spread, runs = oracle_spread(tree, variant, 10000)
    print(variant, "gpu", e_g, "oracle runs", runs)
    assert lo / spread <= e_g <= hi * spread


def test_small_game_vanilla_trajectory(cfr):
    """~450-node game (integer payoffs), vanilla CFR, 1000 iterations,
    exploitability every 100: at every checkpoint one more iteration from the
    GPU's state matches the oracle and both compute the same FP64
    exploitability; the final value lies within the oracle's own spread."""
    tree = G.small_random_game(1)
    s = cfr.Solver(tree)
    for k in range(10):
        s.iterate(99, "cfr")
        check_step_from_gpu_state(s, tree, "cfr")
    e_g = s.exploitability()[0]
    lo, hi, spread, runs = oracle_spread(tree, "cfr", 1000)
    print("small vanilla gpu", e_g, "oracle runs", runs)
    assert lo / spread <= e_g <= hi * spread, (e_g, runs)


def test_batch_game_is_identical_alone_and_in_mix(cfr):
    trees = [G.sized_random_game(1000 + k, 10 ** (2 + (k % 4))) for k in range(8)]
    batch = cfr.Solver(trees)
    batch.iterate(50, "cfr+")
    for g in (0, 3, 7):
        alone = cfr.Solver(trees[g])
        alone.iterate(50, "cfr+")
        for p in (1, 2):
            a = alone.get_state(p)
            b = batch.get_state(p, game=g)
            assert np.array_equal(a["r"], b["r"]) and np.array_equal(a["xbar"], b["xbar"])
            assert np.array_equal(a["b"], b["b"])


def test_many_small_games_keep_their_averages(cfr):
    # more game roots than CTAs: every CTA may end its bottom-up queue on a
    # root, and the average update (Alg. 2) must still cover every sequence
    trees = [G.sized_random_game(5000 + k, 120) for k in range(1500)]
    s = cfr.Solver(trees)
    s.iterate(6, "cfr+")
    for g in (0, 749, 1499):
        alone = cfr.Solver(trees[g])
        alone.iterate(6, "cfr+")
        for p in (1, 2):
            a = alone.get_state(p)
            b = s.get_state(p, game=g)
            assert np.array_equal(a["xbar"], b["xbar"]) and np.array_equal(a["r"], b["r"])


def test_active_mask_freezes_games(cfr):
    trees = [G.sized_random_game(2000 + k, 500) for k in range(4)]
    s = cfr.Solver(trees)
    s.iterate(10, "dcfr", active=[1, 0, 1, 0])
    assert [s.sizes(g)["t"] for g in range(4)] == [10, 0, 10, 0]
    st = s.get_state(1, game=1)
    assert np.all(st["r"] == 0.0)


def test_games_at_different_iterations_advance_independently(cfr):
    # a table whose games hold different counters (each game's own weights
    # t^gamma in the average update, Alg. 4) against each game run alone
    trees = [G.sized_random_game(3000 + k, 10 ** (2 + (k % 3))) for k in range(4)]
    s = cfr.Solver(trees)
    s.iterate(7, "dcfr", active=[1, 1, 0, 0])
    s.iterate(20, "dcfr")
    assert [s.sizes(g)["t"] for g in range(4)] == [27, 27, 20, 20]
    for g, n in ((1, 27), (2, 20)):
        alone = cfr.Solver(trees[g])
        alone.iterate(n, "dcfr")
        for p in (1, 2):
            a = alone.get_state(p)
            b = s.get_state(p, game=g)
            assert np.array_equal(a["r"], b["r"]) and np.array_equal(a["xbar"], b["xbar"])


def test_graph_length_does_not_change_results(cfr):
    tree = G.poker_game()
    a = cfr.Solver(tree)
    b = cfr.Solver(tree)
    a.set_graph_iterations(1)
    b.set_graph_iterations(64)
    a.iterate(130, "pcfr+")
    b.iterate(130, "pcfr+")
    for p in (1, 2):
        assert np.array_equal(a.get_state(p)["r"], b.get_state(p)["r"])


def test_checkpoint_resume(cfr):
    tree = G.poker_game()
    a = cfr.Solver(tree)
    a.iterate(100, "dcfr")
    b = cfr.Solver(tree)
    b.iterate(50, "dcfr")
    c = cfr.Solver(tree)
    for p in (1, 2):
        st = b.get_state(p)
        c.set_state(p, st["r"], st["b"], st["xbar"], st["t"])
    c.iterate(50, "dcfr")
    for p in (1, 2):
        x, y = a.get_state(p), c.get_state(p)
        assert rel(y["r"], x["r"]) < 1e-12 and rel(y["xbar"], x["xbar"]) < 1e-12
        assert x["t"] == y["t"] == 100


def _tree(parent, kind, infoset, action, prob, payoff):
    return G.Tree(np.array(parent, np.int32), np.array(kind, np.int8), np.array(infoset, np.int32),
                  np.array(action, np.int32), np.array(prob, np.float64), np.array(payoff, np.float64))


def degenerate_games():
    return {
        # the root is a terminal: no sequence but the empty one for either player
        "terminal_root": _tree([-1], [3], [-1], [0], [1.0], [2.5]),
        # chance alone decides
        "chance_only": _tree([-1, 0, 0], [0, 3, 3], [-1, -1, -1], [0, 0, 1], [1.0, 0.3, 0.7], [0.0, 1.0, -2.0]),
        # only player 1 decides (player 2 has the empty sequence only)
        "p1_only": _tree([-1, 0, 0, 0], [1, 3, 3, 3], [0, -1, -1, -1], [0, 0, 1, 2], [1.0] * 4, [0.0, 1.0, -2.0, 0.5]),
        # only player 2 decides, below a chance node
        "p2_only": _tree([-1, 0, 0, 1, 1, 2, 2], [0, 2, 2, 3, 3, 3, 3], [-1, 0, 0, -1, -1, -1, -1],
                         [0, 0, 1, 0, 1, 0, 1], [1.0, 0.5, 0.5, 1.0, 1.0, 1.0, 1.0],
                         [0.0, 0.0, 0.0, 1.0, -1.0, 2.0, 0.0]),
    }


@pytest.mark.parametrize("variant", ["cfr", "cfr+", "dcfr", "pcfr+"])
def test_degenerate_games_match_oracle(cfr, variant):
    games = degenerate_games()
    trees = list(games.values()) + [G.poker_game()]
    batch = cfr.Solver(trees)
    batch.iterate(12, variant)
    eb, b1b, b2b = batch.exploitability_batch()
    for k, (name, t) in enumerate(games.items()):
        o = Oracle(t)
        o.iterate(12, variant)
        s = cfr.Solver(t)
        s.iterate(12, variant)
        e_o, b1_o, b2_o = o.exploitability()
        e_g, b1_g, b2_g = s.exploitability()
        # FP32 strategies against the FP64 oracle: exploitability to the
        # suite's relative bar, best-response values to the one-step bar
        for got in ((e_g, b1_g, b2_g), (eb[k], b1b[k], b2b[k])):
            assert abs(got[0] - e_o) <= EXPL_RTOL * abs(e_o) + 1e-9, (name, got, (e_o, b1_o, b2_o))
            assert np.allclose(got[1:], (b1_o, b2_o), rtol=ONE_STEP_RTOL, atol=1e-9), (name, got, (e_o, b1_o, b2_o))
        for p in (1, 2):
            g_, o_ = s.get_state(p), o.get_state(p)
            assert g_["t"] == o_["t"] == 12
            assert np.allclose(g_["r"], o_["r"], rtol=1e-5, atol=1e-6), (name, p)
            assert np.allclose(g_["xbar"], o_["xbar"], rtol=1e-5, atol=1e-6), (name, p)
            a = batch.get_state(p, game=k)
            assert np.array_equal(a["r"], g_["r"]) and np.array_equal(a["xbar"], g_["xbar"]), (name, p)
        s.close()
    batch.close()


def test_invalid_trees_rejected(cfr):
    base = G.small_random_game(1)
    bad = G.Tree(base.parent.copy(), base.kind.copy(), base.infoset.copy(), base.action.copy(),
                 base.chance_prob.copy(), base.payoff.copy())
    bad.chance_prob[1] = 0.9
    with pytest.raises(cfr.CFRError) as e:
        cfr.Solver(bad)
    assert e.value.status == -1
    bad = G.Tree(base.parent.copy(), base.kind.copy(), base.infoset.copy(), base.action.copy(),
                 base.chance_prob.copy(), base.payoff.copy())
    bad.payoff[-1] = np.inf
    with pytest.raises(cfr.CFRError):
        cfr.Solver(bad)


def test_large_game_one_iteration(cfr):
    """depth-12 game, ~6.2e6 nodes, DCFR: one iteration from identical state on
    the full vectors, in the launch configuration the benchmark times."""
    tree = G.large_random_game(3)
    o = Oracle(tree)
    s = cfr.Solver(tree)
    rng = np.random.default_rng(5)
    for p in (1, 2):
        r, b, xb, t = random_state(o, p, rng)
        o.set_state(p, r, b, xb, t)
        s.set_state(p, r, b, xb, t)
    o.iterate(1, "dcfr")
    s.iterate(1, "dcfr")
    for p in (1, 2):
        g_, o_ = s.get_state(p), o.get_state(p)
        assert rel(g_["r"], o_["r"]) <= ONE_STEP_RTOL
        assert rel(g_["xbar"], o_["xbar"]) <= ONE_STEP_RTOL
        assert rel(g_["b"], o_["b"]) <= ONE_STEP_RTOL
    e_o = o.exploitability()
    e_g = s.exploitability()
    assert abs(e_g[0] - e_o[0]) <= 1e-6 * abs(e_o[0])
