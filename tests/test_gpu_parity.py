"""CUDA path (libcfr.so through its C ABI) against the FP64 oracle.

Tolerances:
  * one iteration from identical state: every entry of r, xbar, the next
    sequence-form strategy x and the per-infoset ev within 1e-5 relative
    (element-wise, against max(|oracle entry|, the vector's RMS)); the next
    behavioural strategy b within 1e-5 wherever regret matching's positive
    sum is clearly nonzero;
  * exploitability of identical strategies (FP64 on both sides): 1e-9;
  * final exploitability after T iterations: within 1e-3 relative of the
    oracle's run where the oracle's own summation-order spread is below that
    (stored in tests/golden/trajectory_*.json by make_trajectories.py, which
    calls only the oracle); where the oracle itself spreads wider (integer
    payoffs, near-solved games: Appendix D's divergence), inside the oracle's
    range widened by 1e-3.  Along every trajectory, checkpoints also re-run
    one iteration from the GPU's own state on both sides (1e-5).
"""
import zlib

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2605_14277_b300 import games as G
import json
import os

from tests.parity_util import (EXPL_RTOL, ONE_STEP_RTOL, assert_elementwise, check_ensembles, check_final_expl,
                               oracle_values, random_state, regret_scale, rel, reorder,
                               strategy_mismatch_ok)

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLD, f"trajectory_{name}.json")) as f:
        return json.load(f)

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


def assert_regrets(g_r, o_r, r_old, V, ev, o, p, what):
    sc = regret_scale(o, p, r_old, o_r, V, ev)
    err = np.max(np.abs(g_r - o_r) / np.maximum(sc, 1e-300)) if o_r.size else 0.0
    assert err <= ONE_STEP_RTOL, (what, float(err))


def check_state_and_values(o, s, out, init, alternating, gi=0, what=""):
    """Element-wise parity of r, xbar, b, x and ev after one iteration."""
    vals = oracle_values(o, init, out[1][0]["b"], alternating)
    ev_o = {p: vals[p][1] for p in (1, 2)}
    for p in (1, 2):
        g_, o_ = out[p]
        assert_regrets(g_["r"], o_["r"], init[p][0], vals[p][0], vals[p][1], o, p, ("r", p, what))
        assert_elementwise(g_["xbar"], o_["xbar"], ("xbar", p, what))
        _, na = o.infosets(p)
        assert strategy_mismatch_ok(g_["b"], o_["b"], o_["r"], na) == 0, ("b", p, what)
        v = s.get_values(p, game=gi)
        # the top-down pass: x from the GPU's own next strategy
        assert v["x"][0] == 1.0
        assert_elementwise(v["x"], o.sequence_form(p, g_["b"]), ("x", p, what))
        assert_elementwise(v["ev"], ev_o[p], ("ev", p, what))


def one_step(cfr, tree, variant, mode, seed, game_in_batch=None, **load):
    o = Oracle(tree)
    rng = np.random.default_rng(seed)
    if game_in_batch is None:
        s = cfr.Solver(tree, values=True, **load)
        gi = 0
    else:
        others, gi = game_in_batch
        trees = list(others)
        trees.insert(gi, tree)
        s = cfr.Solver(trees, values=True, **load)
    s.set_update_mode(mode)
    init = {}
    for p in (1, 2):
        r, b, xb, t = random_state(o, p, rng)
        o.set_state(p, r, b, xb, t)
        s.set_state(p, r, b, xb, t, game=gi)
        init[p] = (r, b)
    alt = {"alternating": True, "simultaneous": False}[mode]
    o.iterate(1, variant, alternating=alt)
    s.iterate(1, variant)
    out = {p: (s.get_state(p, game=gi), o.get_state(p)) for p in (1, 2)}
    check_state_and_values(o, s, out, init, alt, gi=gi, what=(tree.name, variant, mode))
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


FP64_RTOL = 1e-11   # precision 64: FP64 on both sides, summation orders differ


@pytest.mark.parametrize("name", ["small_int", "poker", "two_chance"])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("mode", ["alternating", "simultaneous"])
def test_one_iteration_fp64(cfr, name, variant, mode):
    """Precision 64: one iteration from identical state agrees with the
    oracle to rounding (1e-11 element-wise; strategies exactly where regret
    matching's positive sum is not a tie)."""
    tree = parity_games()[name]
    o = Oracle(tree)
    s = cfr.Solver(tree, values=True, precision=64)
    s.set_update_mode(mode)
    rng = np.random.default_rng(zlib.crc32(f"fp64/{name}/{variant}/{mode}".encode()))
    init = {}
    for p in (1, 2):
        r, b, xb, t = random_state(o, p, rng)
        o.set_state(p, r, b, xb, t)
        s.set_state(p, r, b, xb, t)
        init[p] = (r, b)
    alt = mode == "alternating"
    o.iterate(1, variant, alternating=alt)
    s.iterate(1, variant)
    vals = oracle_values(o, init, s.get_state(1)["b"], alt)
    for p in (1, 2):
        g_, o_ = s.get_state(p), o.get_state(p)
        assert g_["t"] == o_["t"] == 6
        for k in ("r", "xbar"):
            assert_elementwise(g_[k], o_[k], (k, p), tol=FP64_RTOL)
        _, na = o.infosets(p)
        assert strategy_mismatch_ok(g_["b"], o_["b"], o_["r"], na, tol=1e-10, tie=1e-12) == 0
        v = s.get_values(p)
        assert v["x"][0] == 1.0
        assert_elementwise(v["x"], o.sequence_form(p, g_["b"]), ("x", p), tol=FP64_RTOL)
        assert_elementwise(v["ev"], vals[p][1], ("ev", p), tol=FP64_RTOL)


@pytest.mark.parametrize("variant,alpha,beta,gamma", [("dcfr", 1.0, 0.5, 3.0), ("dcfr", 2.0, -0.5, 0.0),
                                                      ("pcfr", 0.0, 0.0, 1.5), ("cfr+", 0.0, 0.0, 2.0)])
@pytest.mark.parametrize("mode", ["alternating", "simultaneous"])
def test_one_iteration_other_parameters(cfr, variant, alpha, beta, gamma, mode):
    # non-default discount and averaging exponents (the per-iteration
    # parameter table), one iteration from identical state
    tree = G.random_game(11, depth=8, chance={0: 4, 4: 3}, actions=(2, 3, 4), payoff="normal")
    o = Oracle(tree)
    s = cfr.Solver(tree, values=True)
    s.set_update_mode(mode)
    rng = np.random.default_rng(zlib.crc32(f"{variant}/{alpha}/{beta}/{gamma}/{mode}".encode()))
    init = {}
    for p in (1, 2):
        r, b, xb, t = random_state(o, p, rng)
        o.set_state(p, r, b, xb, t)
        s.set_state(p, r, b, xb, t)
        init[p] = (r, b)
    o.iterate(1, variant, alpha=alpha, beta=beta, gamma=gamma, alternating=(mode == "alternating"))
    s.iterate(1, variant, alpha=alpha, beta=beta, gamma=gamma)
    out = {p: (s.get_state(p), o.get_state(p)) for p in (1, 2)}
    check_state_and_values(o, s, out, init, mode == "alternating", what=(variant, alpha, beta, gamma, mode))


def test_one_iteration_inside_a_batch(cfr):
    others = [G.sized_random_game(40 + k, 10 ** (2 + k % 3)) for k in range(5)]
    tree = G.poker_game()
    for variant in VARIANTS:
        one_step(cfr, tree, variant, "alternating", seed=3, game_in_batch=(others, 2))


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


def check_step_from_gpu_state(s, trees, variant, games=(0,), oracle=None):
    """For each listed game of the solver: both sides compute the FP64
    exploitability of the GPU's current averages (1e-9), then run one more
    iteration from the GPU's state (element-wise 1e-5; only that game is
    advanced on the GPU).  Returns the GPU's exploitabilities (game order)."""
    trees = trees if isinstance(trees, list) else [trees]
    out = []
    for gi in games:
        o = oracle if oracle is not None else Oracle(trees[gi])
        for p in (1, 2):
            st = s.get_state(p, game=gi)
            o.set_state(p, st["r"], st["b"], st["xbar"], st["t"])
        e_o, b1_o, b2_o = o.exploitability()
        eb, b1b, b2b = s.exploitability_batch()
        e_g, b1_g, b2_g = eb[gi], b1b[gi], b2b[gi]
        assert abs(b1_g - b1_o) <= 1e-9 * max(1.0, abs(b1_o)) and abs(b2_g - b2_o) <= 1e-9 * max(1.0, abs(b2_o))
        out.append(e_g)
        init = {p: (o.get_state(p)["r"], o.get_state(p)["b"]) for p in (1, 2)}
        o.iterate(1, variant)
        if s.n_games == 1:
            s.iterate(1, variant)
        else:
            s.iterate(1, variant, active=[1 if g == gi else 0 for g in range(s.n_games)])
        b1_next = s.get_state(1, game=gi)["b"]
        vals = oracle_values(o, init, b1_next, alternating=(variant != "cfr"))
        for p in (1, 2):
            g_, o_ = s.get_state(p, game=gi), o.get_state(p)
            for k in ("r", "b", "xbar"):
                assert np.isfinite(g_[k]).all(), (k, p, gi)
            assert_regrets(g_["r"], o_["r"], init[p][0], vals[p][0], vals[p][1], o, p, ("r", p, gi))
            assert_elementwise(g_["xbar"], o_["xbar"], ("xbar", p, gi))
            _, na = o.infosets(p)
            assert strategy_mismatch_ok(g_["b"], o_["b"], o_["r"], na) == 0
    return out


GPU_REORDERS = 8   # GPU runs on reordered copies for the end-value ensembles


def gpu_end_values(cfr, tree, variant, T, e_base, n_reorder=GPU_REORDERS, make=None):
    """Exploitability after T iterations of the GPU on the game (e_base, from
    the trajectory) and on its first n_reorder reorderings (the same
    `reorder` seeds as the oracle's stored runs)."""
    runs = {"base": e_base}
    for k in range(1, n_reorder + 1):
        g = (make or cfr.Solver)(reorder(tree, k))
        g.iterate(T, variant)
        runs[f"reorder{k}"] = g.exploitability()[0]
        g.close()
    return runs


def run_trajectory(cfr, s, tree, variant, checkpoints, gold, o=None, n_reorder=GPU_REORDERS, make=None):
    """Iterate to each checkpoint and re-synchronise one step from the GPU's
    state there (both sides also compute the same FP64 exploitability of the
    GPU's averages); at the last checkpoint, the end of the run, compare the
    GPU's exploitability ensemble with the oracle's stored runs
    (check_ensembles).  Returns the exploitabilities seen (for the report)."""
    done, report = 0, []
    for k, c in enumerate(checkpoints):
        s.iterate(c - done, variant)
        e_g = check_step_from_gpu_state(s, tree, variant, oracle=o)[0]
        runs = {name: r[k] for name, r in gold.items()}
        vals = list(runs.values())
        so = max(vals) / min(vals) - 1.0
        err = abs(e_g - runs["base"]) / runs["base"]
        row = (c, e_g, runs["base"], err, so, None, "resync")
        if k == len(checkpoints) - 1:
            g_runs = gpu_end_values(cfr, tree, variant, c, e_g, n_reorder, make)
            kind, err, so, sg = check_ensembles(g_runs, runs, (tree.name, variant, c))
            row = (c, e_g, runs["base"], err, so, sg, kind)
        report.append(row)
        done = c + 1
    return report


def print_report(label, report):
    for c, e_g, e_o, err, so, sg, kind in report:
        gs = "" if sg is None else f" gpu spread {sg:.2e}"
        print(f"{label} t={c}: gpu {e_g:.9e} oracle {e_o:.9e} rel err {err:.2e} "
              f"oracle spread {so:.2e}{gs} -> {kind}")


@pytest.mark.parametrize("variant", ["cfr+", "dcfr", "pcfr+", "pcfr"])
def test_poker_trajectory_10k(cfr, variant):
    """Poker (integer payoffs), 10^4 iterations: one iteration from the GPU's
    state matches the oracle at t = 1000, 5000 and 10^4; the end value against
    the oracle's stored runs (check_ensembles)."""
    gold = golden("poker")
    tree = G.poker_game()
    s = cfr.Solver(tree)
    report = run_trajectory(cfr, s, tree, variant, gold["checkpoints"], gold["variants"][variant])
    print_report(f"poker {variant}", report)


def test_small_game_vanilla_trajectory_fp64(cfr):
    """~450-node game whose payoffs are given in FP64, vanilla CFR, 1000
    iterations in precision 64, exploitability every 100: one more iteration
    from the GPU's state matches the oracle at each checkpoint, and the end
    value is within 1e-3 of the oracle's (whose own summation-order spread
    is ~1e-10 here)."""
    gold = golden("small_cfr")
    tree = G.small_random_game(1)
    s = cfr.Solver(tree, precision=64)

    def make(t):
        return cfr.Solver(t, precision=64)

    report = run_trajectory(cfr, s, tree, "cfr", gold["checkpoints"], gold["runs"], make=make)
    print_report("small cfr fp64", report)
    assert report[-1][-1] == "bound"


def test_small_game_vanilla_trajectory_fp32(cfr):
    """The same game with FP32 passes: every checkpoint's one-step resync
    matches the oracle.  The end value is reported, not bounded: at t = 1 two
    of player 2's actions tie exactly (the FP64 oracle's regrets are 0 and 0,
    uniform next strategy) while FP32 rounding leaves them at -2^-30 and
    +2^-30 (a pure next strategy), so the two trajectories part at once
    (the regret-matching sensitivity of Appendix D); precision 64 removes it."""
    gold = golden("small_cfr")
    tree = G.small_random_game(1)
    s = cfr.Solver(tree)
    done = 0
    for c in gold["checkpoints"]:
        s.iterate(c - done, "cfr")
        e_g = check_step_from_gpu_state(s, tree, "cfr")[0]
        done = c + 1
    e_o = gold["runs"]["base"][-1]
    print(f"small cfr fp32 t={gold['checkpoints'][-1]}: gpu {e_g:.9e} oracle {e_o:.9e} rel err {abs(e_g - e_o) / e_o:.2e}")


def test_large_game_dcfr_trajectory_10k(cfr):
    """The 6.2M-node game, DCFR(1.5, 0, 2), 10^4 iterations through the graph
    path (64-iteration CUDA graphs): one iteration from the GPU's state
    matches the oracle at t = 1000, 5000 and 10^4; the end value against the
    oracle's stored runs (check_ensembles, two reorderings a side)."""
    gold = golden("large_dcfr")
    tree = G.large_random_game(3)
    s = cfr.Solver(tree)
    o = Oracle(tree)
    report = run_trajectory(cfr, s, tree, "dcfr", gold["checkpoints"], gold["runs"], o=o, n_reorder=2)
    print_report("large dcfr", report)


def test_batch_sample_trajectory(cfr):
    """64 games of the 4096-game batch at their own sizes in one context,
    CFR+, 1024 iterations as 16 replays of a 64-iteration CUDA graph: each
    game's exploitability against the oracle's stored runs (check_ensembles,
    with the GPU's runs on eight reorderings of every game, batched into a
    second context); then one more iteration from the GPU's state on both
    sides for four of the games."""
    gold = golden("batch_cfrplus")
    seeds = [int(k) for k in gold["games"]]
    trees = [G.batch_game(sd) for sd in seeds]
    T = gold["checkpoints"][-1]
    rtrees = [reorder(t, k) for t in trees for k in range(1, GPU_REORDERS + 1)]
    for prec in (32, 64):
        s = cfr.Solver(trees, precision=prec)
        s.iterate(T, "cfr+")
        eb = s.exploitability_batch()[0]
        r = cfr.Solver(rtrees, precision=prec)
        r.iterate(T, "cfr+")
        er = r.exploitability_batch()[0].reshape(len(trees), GPU_REORDERS)
        r.close()
        kinds = {"bound": 0, "ranges overlap": 0, "fail": 0}
        worst, errs, fails = 0.0, [], []
        for gi, sd in enumerate(seeds):
            runs = {name: v[-1] for name, v in gold["games"][str(sd)].items()}
            g_runs = {"base": eb[gi], **{f"reorder{k + 1}": er[gi, k] for k in range(GPU_REORDERS)}}
            try:
                kind, err, so, sg = check_ensembles(g_runs, runs, ("batch", sd))
            except AssertionError:
                kind, err = "fail", abs(eb[gi] - runs["base"]) / runs["base"]
                fails.append((sd, float(err)))
            kinds[kind] += 1
            errs.append(err)
            if kind == "bound":
                worst = max(worst, err)
        print(f"batch sample, precision {prec}: {kinds['bound']} games at the 1e-3 bound (worst rel err "
              f"{worst:.2e}), {kinds['ranges overlap']} rounding-sensitive games with overlapping ranges, "
              f"{kinds['fail']} outside {fails}; median rel err of the base runs {np.median(errs):.2e}")
        # FP64 passes: every game; FP32 passes: all but a few games whose
        # iterates FP32 rounding or range moves (the reason precision 64 exists)
        assert kinds["fail"] <= (0 if prec == 64 else len(seeds) // 10), fails
        check_step_from_gpu_state(s, trees, "cfr+", games=(0, 17, 40, 63))
        s.close()


def test_tiny_counterfactual_values_stay_finite(cfr):
    """Regrets scale with the opponent's reach and can fall below FP32's
    normal range once strategies sharpen deep in a game.  Poker with payoffs
    scaled by 2^-120 puts every value there from the start: regret matching
    must still give finite strategies on each simplex (the normaliser of a
    tiny positive sum would otherwise overflow), and the FP64 exploitability
    must scale with the payoffs."""
    base = G.poker_game()
    tiny = G.Tree(base.parent, base.kind, base.infoset, base.action, base.chance_prob,
                  base.payoff * 2.0 ** -120)
    a, b = cfr.Solver(base), cfr.Solver(tiny)
    a.iterate(300, "dcfr")
    b.iterate(300, "dcfr")
    o = Oracle(tiny)
    for p in (1, 2):
        st = b.get_state(p)
        for k in ("r", "b", "xbar"):
            assert np.isfinite(st[k]).all(), (k, p)
        _, na = o.infosets(p)
        sums = np.add.reduceat(st["b"], np.r_[0, np.cumsum(na)[:-1]])
        assert np.allclose(sums, 1.0, atol=1e-5) and (st["b"] >= 0).all()
    e_a, e_b = a.exploitability()[0], b.exploitability()[0]
    assert np.isfinite(e_b) and e_b > 0
    assert 0.5 < (e_b * 2.0 ** 120) / e_a < 2.0, (e_a, e_b * 2.0 ** 120)


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


def test_prepared_graph_replays_the_same_iterations(cfr):
    """prepare_graph captures without running: the state stays put, and the
    iterations replayed from the prepared graph equal eager ones."""
    tree = G.poker_game()
    a = cfr.Solver(tree)
    b = cfr.Solver(tree)
    a.set_graph_iterations(1)
    b.set_graph_iterations(20)
    before = b.get_state(1)["r"].copy()
    b.prepare_graph("dcfr")
    b.prepare_graph("pcfr+")
    b.sync()
    assert np.array_equal(b.get_state(1)["r"], before)
    assert b.sizes(0)["t"] == 0
    a.iterate(40, "dcfr")
    b.iterate(40, "dcfr")
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
    s = cfr.Solver(tree, values=True)
    rng = np.random.default_rng(5)
    init = {}
    for p in (1, 2):
        r, b, xb, t = random_state(o, p, rng)
        o.set_state(p, r, b, xb, t)
        s.set_state(p, r, b, xb, t)
        init[p] = (r, b)
    o.iterate(1, "dcfr")
    s.iterate(1, "dcfr")
    out = {p: (s.get_state(p), o.get_state(p)) for p in (1, 2)}
    check_state_and_values(o, s, out, init, True, what="large")
    for p in (1, 2):
        assert_elementwise(out[p][0]["b"], out[p][1]["b"], ("b", p))
    e_o = o.exploitability()
    e_g = s.exploitability()
    assert abs(e_g[0] - e_o[0]) <= 1e-6 * abs(e_o[0])
