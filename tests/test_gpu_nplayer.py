"""n-player CUDA path (libcfr.so's cfrn_* entry points) against the n-player FP64
oracle (oracle/nplayer.py, pinned in test_nplayer_oracle.py).

Tolerances, read as in the two-player suite (test_gpu_parity.py):
  * one iteration from identical state (the oracle loaded with the GPU's r, b,
    xbar): every regret within 1e-5 of the size of its update (|r_old| plus
    V and ev recomputed over the absolute values of the payoff terms -- the
    magnitudes the FP32 sums run over, which cancellation in V and ev can
    hide -- or the vector's RMS if larger); every xbar entry
    within 1e-5 (against max(|entry|, the vector's RMS)); the next behavioural
    strategy within 1e-5 wherever regret matching's positive sum is clearly
    nonzero (elsewhere only its validity); the next x, rebuilt from the GPU's
    own b, within 1e-5;
  * the tensor contraction u_i against the other players' current x (as the
    GPU holds them): within 1e-5 of sum_e |val_e prod_k x_k| per sequence (FP32
    products and sums against FP64) or the vector's RMS;
  * NashConv of identical averages (FP64 on both sides): 1e-9 relative;
  * after T iterations from the start, NashConv within 1e-3 relative of the
    oracle's own run on games with continuous payoffs.
"""
import numpy as np
import pytest

from oracle.nplayer import CFR, CFR_PLUS, DCFR, NGame, NOracle, PCFR, PCFR_PLUS
from paper_2605_14277_b300 import games as G

pytestmark = pytest.mark.gpu

VARIANTS = {"cfr": (CFR, (0.0, 0.0, 0.0)), "cfr+": (CFR_PLUS, (0.0, 0.0, 1.0)), "dcfr": (DCFR, (1.5, 0.0, 2.0)),
            "pcfr+": (PCFR_PLUS, (0.0, 0.0, 2.0)), "pcfr": (PCFR, (0.0, 0.0, 0.0))}
TOL = 1e-5


@pytest.fixture(scope="module")
def NP():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_14277_b300 import nplayer
    return nplayer


def games():
    return {
        "kuhn3": G.kuhn3_game(),
        "small3": G.small_nplayer_game(3, 1),
        "four": G.random_nplayer_game(4, 7, depth=8, chance={0: 3, 4: 2}, actions=(2, 3)),
        "five_general_sum": G.random_nplayer_game(5, 3, depth=6, chance={0: 2}, actions=(2, 3), zero_sum=False),
        "two_in_three": G.nplayer_from_two_player(G.small_random_game(1), 3),
        # six players: the first three have levels of ~110 child decision
        # points per sequence (worked a warp per decision point), the last
        # three tensor rows of 32 and more entries (a warp per row)
        "six_wide": G.random_nplayer_game(6, 11, depth=10, chance={0: 3}, actions=(2, 3)),
    }


def oracle_from_gpu(tree, s):
    o = NOracle(tree)
    for i in range(tree.n_players):
        st = s.get_state(i)
        o.r[i][1:] = st["r"]
        o.b[i][1:] = st["b"]
        o.xbar[i] = st["xbar"].copy()
        o.t = st["t"]
    return o


def elementwise(g, o, scale):
    g, o = np.asarray(g, np.float64), np.asarray(o, np.float64)
    if o.size == 0:
        return 0.0
    den = np.maximum(np.abs(o), np.maximum(scale, np.sqrt(np.mean(o * o))))
    return float(np.max(np.abs(g - o) / np.maximum(den, 1e-300)))


def strategies_match(P, b_gpu, b_orc, rm_input, r_scale):
    """Infoset by infoset, the next behavioural strategies.  Regret matching
    b = q / sum(q), q = (input)^+, moves by at most 2 delta / sum(q) when each
    input moves by delta, and the inputs are held to delta = TOL * (their
    update's scale): so b must agree within TOL + 2 delta / sum(q), which
    reduces to a validity check (a distribution) when sum(q) is at the
    rounding level.  Returns the offending infosets."""
    bad = []
    if P.J == 0:
        return bad
    q = np.maximum(rm_input, 0.0)
    pos = np.add.reduceat(q, P.off - 1)
    dmax = np.maximum.reduceat(TOL * r_scale, P.off - 1)
    tol = TOL + 2.0 * dmax / np.maximum(pos, 1e-300)
    diff = np.maximum.reduceat(np.abs(b_gpu - b_orc), P.off - 1)
    sums = np.add.reduceat(b_gpu, P.off - 1)
    assert (np.abs(sums - 1.0) < 1e-5).all() and (b_gpu >= 0).all()
    for j in np.flatnonzero(diff > tol):
        sl = slice(P.off[j] - 1, P.off[j] - 1 + P.nact[j])
        bad.append((int(j), b_gpu[sl].tolist(), b_orc[sl].tolist(), rm_input[sl].tolist(), float(tol[j])))
    return bad


def abs_utility(game, i, xs):
    """sum over entries of |pi_c payoff_i prod_k x_k| per sequence (the scale of u_i's rounding)"""
    prod = np.abs(game.treach * game.tpay[:, i])
    for k in range(game.n):
        if k != i:
            prod = prod * np.abs(xs[k][game.tseq[:, k]])
    u = np.zeros(game.pl[i].S + 1)
    np.add.at(u, game.tseq[:, i], prod)
    return u


def check_one_step(s, tree, variant, alternating, what="", params=None):
    """One iteration from the GPU's state: the GPU's, against the step the
    oracle's primitives take from the same state, element-wise.  params:
    (alpha, beta, gamma) instead of the variant's defaults."""
    v, (a, b, g) = VARIANTS[variant]
    if params is not None:
        a, b, g = params
    n = tree.n_players
    o = oracle_from_gpu(tree, s)
    game = o.g
    # the contraction against the GPU's current x
    xg = [s.get_values(i)[0] for i in range(n)]
    for i in range(n):
        u_g = s.get_values(i)[1]
        u_o = game.utility(i, xg)
        assert elementwise(u_g, u_o, abs_utility(game, i, xg)) <= TOL, ("u", i, what)
    init = [(o.r[i].copy(), o.b[i].copy(), o.xbar[i].copy()) for i in range(n)]
    tt = float(o.t + 1)
    s.iterate(1, variant, alpha=a, beta=b, gamma=g, alternating=alternating)
    out = [s.get_state(i) for i in range(n)]
    # The oracle's step for each player, from the oracle's own primitives
    # (Alg. 1 ObserveUtility, the post-op, regret matching, the average):
    # under alternating updates the players before i are taken at the GPU's
    # next strategy, so that a regret-matching decision upstream that rounding
    # tipped cannot leak into player i's check.
    xs0 = [NGame.sequence_form(P, init[i][1]) for i, P in enumerate(game.pl)]
    for i, P in enumerate(game.pl):
        xs = list(xs0)
        if alternating:
            for k in range(i):
                xs[k] = NGame.sequence_form(game.pl[k], np.concatenate([[0.0], out[k]["b"]]))
        u = game.utility(i, xs)
        r_exp = init[i][0].copy()
        V, ev = NGame.observe_utility(P, u, init[i][1], r_exp)
        NGame.post_op(r_exp, v, tt, a, b)
        d = V[1:] - ev[P.seq_inf] if P.J else np.zeros(0)
        rm_in = r_exp.copy()
        if v in (PCFR_PLUS, PCFR):            # NextStrategy*(m = u): RM of r + the observed regret
            rm_in[1:] += d
        b_exp = NGame.regret_matching(P, rm_in)
        xbar_exp = init[i][2] + tt ** g * xs0[i]
        # the magnitudes the FP32 sums run over: the same bottom-up pass on
        # |terms| (V and ev can cancel far below them)
        Va, eva = NGame.observe_utility(P, abs_utility(game, i, xs), init[i][1], init[i][0].copy())
        g_ = out[i]
        for k in ("r", "b", "xbar"):
            assert np.isfinite(g_[k]).all(), (k, i, what)
        scale = np.abs(init[i][0][1:]) + Va[1:] + (eva[P.seq_inf] if P.J else 0.0)
        r_o = r_exp[1:]
        sc = np.zeros(0)
        if r_o.size:
            sc = np.maximum(scale, np.sqrt(np.mean(r_o * r_o)))
            err = float(np.max(np.abs(g_["r"] - r_o) / np.maximum(sc, 1e-300)))
            assert err <= TOL, ("r", i, what, err)
        assert elementwise(g_["xbar"], xbar_exp, 0.0) <= TOL, ("xbar", i, what)
        bad = strategies_match(P, g_["b"], b_exp[1:], rm_in[1:], 2.0 * sc if v in (PCFR_PLUS, PCFR) else sc)
        assert bad == [], ("b", i, what, bad[:3])
        x_g = s.get_values(i)[0]
        assert x_g[0] == 1.0
        x_o = NGame.sequence_form(P, np.concatenate([[0.0], g_["b"]]))
        assert elementwise(x_g, x_o, 0.0) <= TOL, ("x", i, what)


@pytest.mark.parametrize("variant", sorted(VARIANTS))
@pytest.mark.parametrize("alternating", [True, False])
def test_one_step_parity(NP, variant, alternating):
    for name, tree in games().items():
        s = NP.NSolver(tree)
        check_one_step(s, tree, variant, alternating, (name, "t=0"))
        s.iterate(6, variant, alternating=alternating)
        check_one_step(s, tree, variant, alternating, (name, "t=7"))
        s.close()


def test_nash_conv_of_identical_averages(NP):
    for name, tree in games().items():
        s = NP.NSolver(tree)
        # t = 0: no average yet, so the current strategies, the GPU's FP32 x
        # on both sides
        nc0, g0 = s.nash_conv()
        o = NOracle(tree)
        nco, go = o.nash_conv([s.get_values(i)[0] for i in range(tree.n_players)])
        assert nc0 == pytest.approx(nco, rel=1e-9, abs=1e-12), name
        s.iterate(30, "dcfr")
        o = oracle_from_gpu(tree, s)
        nc, gains = s.nash_conv()
        nco, go = o.nash_conv()
        assert nc == pytest.approx(nco, rel=1e-9, abs=1e-12), name
        for i in range(tree.n_players):
            assert gains[i] == pytest.approx(go[i], rel=1e-9, abs=1e-12), (name, i)
            assert gains[i] >= -1e-9                  # a best response is never worse
        s.close()


def test_graph_length_does_not_change_results(NP):
    tree = G.small_nplayer_game(3, 2)
    states = []
    for k in (1, 7, 64):
        s = NP.NSolver(tree)
        s.set_graph_iterations(k)
        s.iterate(100, "pcfr+")
        states.append([s.get_state(i) for i in range(3)])
        assert s.t == 100
        s.close()
    for other in states[1:]:
        for a, b in zip(states[0], other):
            for key in ("r", "b", "xbar"):
                assert np.array_equal(a[key], b[key])


def test_player_who_never_acts_changes_nothing(NP):
    """A two-player game with a third player who never acts: the same bits as
    the game given with two players (the extra factor x[empty] = 1 is exact)."""
    base = G.small_random_game(2)
    s2 = NP.NSolver(G.nplayer_from_two_player(base, 2))
    s3 = NP.NSolver(G.nplayer_from_two_player(base, 3))
    for s in (s2, s3):
        s.iterate(50, "dcfr")
    for i in range(2):
        a, b = s2.get_state(i), s3.get_state(i)
        for key in ("r", "b", "xbar"):
            assert np.array_equal(a[key], b[key])
    nc2, _ = s2.nash_conv()
    nc3, g3 = s3.nash_conv()
    assert nc3 == pytest.approx(nc2, rel=1e-12) and g3[2] == pytest.approx(0.0, abs=1e-12)


def test_two_player_games_agree_with_the_two_player_path(NP):
    """The same two-player game through the two-player kernels and through the
    n-player ones: one iteration from the start agrees element-wise."""
    from paper_2605_14277_b300 import cfr as C
    tree = G.random_game(1, depth=6, chance={0: 3}, actions=(2, 3), payoff="normal")
    s2 = C.Solver(tree)
    sn = NP.NSolver(G.nplayer_from_two_player(tree, 2))
    for it in (1, 2):
        s2.iterate(1, "cfr+")
        sn.iterate(1, "cfr+")
        for p in (1, 2):
            a, b = s2.get_state(p), sn.get_state(p - 1)
            assert elementwise(b["r"], a["r"], 0.0) <= TOL and elementwise(b["xbar"], a["xbar"], 0.0) <= TOL


@pytest.mark.parametrize("name,variant,checkpoints", [("small3", "dcfr", (30, 80)), ("four", "cfr+", (100, 400)),
                                                      ("five_general_sum", "pcfr+", (30, 80))])
def test_trajectory_end_value(NP, name, variant, checkpoints):
    """T iterations from the start on both sides: checkpoints re-run one
    iteration from the GPU's state, and the final NashConv of the GPU's
    averages is within 1e-3 relative of the oracle's own run.  The runs stop
    while NashConv is above 1e-5 of the payoff range: nearer a solution the
    FP32 passes' rounding (about 1e-8 of the range in NashConv) is what is
    left of the difference (the divergence Appendix D reports)."""
    tree = games()[name]
    v, (a, b, g) = VARIANTS[variant]
    s = NP.NSolver(tree)
    done = 0
    for c in checkpoints:
        s.iterate(c - done, variant)
        done = c
        check_one_step(s, tree, variant, True, (name, c))
        done += 1
    o = NOracle(tree)
    o.iterate(done, v, a, b, g)
    nc_g, _ = s.nash_conv()
    nc_o, _ = o.nash_conv()
    assert nc_o > 1e-5 * tree.payoff_range(), (name, nc_o)
    assert abs(nc_g - nc_o) <= 1e-3 * nc_o, (name, nc_g, nc_o)
    s.close()


def test_degenerate_games(NP):
    # a terminal root: nobody acts
    t = G.NTree(3, np.array([-1]), np.array([G.N_TERMINAL]), np.array([-1]), np.array([-1]), np.array([-1]),
                np.array([1.0]), np.array([[1.0, -2.0, 1.0]]))
    s = NP.NSolver(t)
    s.iterate(5, "dcfr")
    nc, gains = s.nash_conv()
    assert nc == 0.0 and (gains == 0.0).all()
    st = s.get_state(0)
    assert st["r"].size == 0 and st["xbar"].shape == (1,) and st["t"] == 5
    s.close()
    # single-action infosets and the largest player count
    t8 = G.random_nplayer_game(8, 4, depth=9, chance={0: 2}, actions=(1, 2), zero_sum=False)
    s = NP.NSolver(t8)
    check_one_step(s, t8, "dcfr", True, "eight players")
    s.iterate(20, "dcfr")
    check_one_step(s, t8, "dcfr", False, "eight players, t=21")
    o = oracle_from_gpu(t8, s)
    assert s.nash_conv()[0] == pytest.approx(o.nash_conv()[0], rel=1e-9, abs=1e-12)
    s.close()


def ladder_game(n, width, depth, split, seed):
    """A deep perfect-information game: a chance deal of `width`, then the
    players take turns (0, 1, ..., n-1, 0, ...) to stop (a terminal with N(0,1)
    payoffs) or go on, for `depth` turns, with a chance split of two after turn
    `split`.  Every player has depth / n levels: the first ones of `width`
    decision points, the rest of 2 * width."""
    rng = np.random.default_rng(seed)
    parent, kind, actor, infoset, action, cprob = [-1], [G.N_CHANCE], [-1], [-1], [-1], [1.0]
    n_inf = [0] * n

    def add(par, k, who, act, p):
        parent.append(par)
        kind.append(k)
        actor.append(who)
        infoset.append(-1)
        action.append(act)
        cprob.append(p)
        return len(parent) - 1

    heads = [add(0, G.N_DECISION, 0, e, 1.0 / width) for e in range(width)]
    for step in range(depth):
        who = step % n
        nxt = []
        for h in heads:
            kind[h], actor[h] = G.N_DECISION, who
            infoset[h] = n_inf[who]
            n_inf[who] += 1
            add(h, G.N_TERMINAL, -1, 0, 1.0)
            if step == depth - 1:
                add(h, G.N_TERMINAL, -1, 1, 1.0)
            elif step == split:
                c = add(h, G.N_CHANCE, -1, 1, 1.0)
                nxt += [add(c, G.N_DECISION, -1, e, 0.5) for e in range(2)]
            else:
                nxt.append(add(h, G.N_DECISION, -1, 1, 1.0))
        heads = nxt
    kind = np.array(kind, np.int8)
    pay = np.where((kind == G.N_TERMINAL)[:, None], rng.standard_normal((len(kind), n)).astype(np.float32), 0.0)
    pay[:, n - 1] = -pay[:, : n - 1].sum(axis=1)
    return G.NTree(n, np.array(parent), kind, np.array(actor), np.array(infoset), np.array(action),
                   np.array(cprob), pay.astype(np.float64))


def test_deep_players_take_the_level_by_level_top_down(NP):
    """Players with more than 17 levels build x level by level (the merged top
    levels in one launch, the wider ones a launch each) instead of in one
    walking launch; both agree with the oracle."""
    tree = ladder_game(3, 1500, 60, 29, 4)
    s = NP.NSolver(tree)
    assert all(sz["levels"] == 20 for sz in s.sizes)
    check_one_step(s, tree, "dcfr", True, "ladder")
    s.iterate(10, "pcfr+")
    check_one_step(s, tree, "pcfr+", False, "ladder, t=11")
    o = oracle_from_gpu(tree, s)
    assert s.nash_conv()[0] == pytest.approx(o.nash_conv()[0], rel=1e-9, abs=1e-12)
    s.close()


def test_level_sizes_match_the_oracle_levels(NP):
    """cfrn_level_sizes: decision points and sequences per level, against the
    oracle's own level numbering of each player's sequence form."""
    for name, tree in games().items():
        s = NP.NSolver(tree)
        g = NGame(tree)
        for i, P in enumerate(g.pl):
            want = [(len(js), len(P.seqs_of(js))) for js in P.levels]
            assert s.level_sizes(i) == want, (name, i)
        s.close()


def test_large_game_one_step(NP):
    """The 4.8M-node three-player game: one iteration from the GPU's state at
    t = 3 against the oracle on the full vectors."""
    tree = G.large_nplayer_game(3)
    s = NP.NSolver(tree)
    s.iterate(3, "dcfr")
    check_one_step(s, tree, "dcfr", True, "large")
    s.close()


def test_five_player_large_game_one_step(NP):
    """The 4.06M-node five-player game at t = 3 against the oracle on the full
    vectors: its players' rows take every row path (player 0, 95k rows of
    17 entries: 8 lanes a row; player 1, 8.8 entries: 4 lanes; players 2-3,
    one thread a row; player 4 and part of player 0, rows of 32 and more
    entries: a warp each)."""
    tree = G.large_nplayer_game(5)
    game = NGame(tree)
    avg = [np.bincount(game.tseq[:, i], minlength=P.S + 1) for i, P in enumerate(game.pl)]
    short = [c[c < 32] for c in avg]
    assert 16 <= short[0].mean() and len(short[0]) > 2048 and 8 <= short[1].mean() < 16
    s = NP.NSolver(tree)
    s.iterate(3, "dcfr")
    check_one_step(s, tree, "dcfr", True, "large, five players")
    s.close()


def test_launch_count(NP):
    tree = G.small_nplayer_game(3, 1)
    s = NP.NSolver(tree)
    L = [s.sizes[i]["levels"] for i in range(3)]
    per_iter = s.sizes[0]["kernels_per_iteration"]
    # every player: rows (with the average update), then its bottom-up and
    # top-down levels, the small top levels merged into one launch each way
    assert 3 + 2 * 3 <= per_iter <= sum(1 + 2 * l for l in L)
    before = s.launches
    s.set_graph_iterations(16)
    s.prepare_graph("dcfr")
    assert s.launches == before          # capturing runs nothing
    s.iterate(32, "dcfr")
    s.sync()
    assert s.launches - before == 32 * per_iter + 2 * 2   # plus a parameter fill and a tick per graph
    s.close()


def test_checkpoint_resume(NP):
    """A context resumed from another's state continues with the same bits;
    a state taken from the oracle gives one-step parity."""
    tree = G.small_nplayer_game(3, 1)
    a = NP.NSolver(tree)
    a.iterate(30, "pcfr+")
    b = NP.NSolver(tree)
    for i in range(3):
        st = a.get_state(i)
        b.set_state(i, st["r"], st["b"], st["xbar"], st["t"])
    assert b.t == 30
    for i in range(3):
        xa, xb = a.get_values(i)[0], b.get_values(i)[0]
        assert np.array_equal(xa, xb)
    a.iterate(20, "pcfr+")
    b.iterate(20, "pcfr+")
    for i in range(3):
        sa, sb = a.get_state(i), b.get_state(i)
        for key in ("r", "b", "xbar"):
            assert np.array_equal(sa[key], sb[key]), key
    # the oracle's state after 15 iterations, resumed on the GPU
    o = NOracle(tree)
    o.iterate(15, DCFR, 1.5, 0.0, 2.0)
    c = NP.NSolver(tree)
    for i in range(3):
        c.set_state(i, o.r[i][1:], o.b[i][1:], o.xbar[i], o.t)
    check_one_step(c, tree, "dcfr", True, "resumed from the oracle")
    # refused: a strategy that is not a distribution
    bad = a.get_state(0)["b"].copy()
    bad[0] += 0.5
    from paper_2605_14277_b300.cfr import CFRError
    with pytest.raises(CFRError):
        a.set_state(0, b=bad)


@pytest.mark.parametrize("variant,params", [("dcfr", (1.0, 0.5, 3.0)), ("dcfr", (2.0, -0.5, 0.0)),
                                            ("cfr+", (0.0, 0.0, 2.0)), ("pcfr", (0.0, 0.0, 1.5))])
def test_nondefault_parameters(NP, variant, params):
    """Non-default DCFR discounts and averaging exponents, both schedules."""
    for name in ("kuhn3", "four"):
        tree = games()[name]
        for alternating in (True, False):
            s = NP.NSolver(tree)
            s.iterate(5, variant, *params, alternating=alternating)
            check_one_step(s, tree, variant, alternating, (name, params), params=params)
            s.close()
