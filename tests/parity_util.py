"""Shared helpers for the GPU-vs-oracle parity tests (inputs and comparisons only)."""
import numpy as np

# one iteration from identical state: relative error per element (see elementwise)
ONE_STEP_RTOL = 1e-5
# final exploitability after T iterations (see test_gpu_parity for the reading)
EXPL_RTOL = 1e-3


def rel(a, b):
    """Norm-wise relative error ||a - b||_2 / ||b||_2 (reported beside the
    element-wise figure; the tests assert element-wise)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = max(np.linalg.norm(b), 1e-300)
    return float(np.linalg.norm(a - b) / den)


def elementwise(g, o, scale=None):
    """Largest element-wise error max_k |g_k - o_k| / max(|o_k|, s), where s is
    the vector's own scale (the RMS of o unless given): a few wrong entries
    cannot hide in the norm of a long vector, and entries near zero are
    measured against the vector's typical size instead of their own."""
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    assert g.shape == o.shape, (g.shape, o.shape)
    if o.size == 0:
        return 0.0
    s = float(np.sqrt(np.mean(o * o))) if scale is None else float(scale)
    den = np.maximum(np.abs(o), max(s, 1e-300))
    return float(np.max(np.abs(g - o) / den))


def assert_elementwise(g, o, what, tol=ONE_STEP_RTOL, scale=None):
    err = elementwise(g, o, scale)
    assert err <= tol, (what, err, rel(g, o))
    return err


def check_ensembles(gpu_runs, oracle_runs, what, rtol=EXPL_RTOL):
    """Final exploitability of a rounding-sensitive run, GPU against oracle.
    Both sides ran the same game and its summation-order reorderings
    (`reorder`); each ensemble's spread is its own sensitivity to rounding
    (FP32 passes on the GPU, FP64 in the oracle; Appendix D).  Where both
    ensembles are tighter than rtol, the GPU's run on the game itself must be
    within rtol of the oracle's (the bound); otherwise the two ranges,
    each widened by rtol, must overlap.  Returns (kind, relative error of
    the two `base` runs, oracle spread, GPU spread)."""
    og = [float(v) for v in oracle_runs.values()]
    gg = [float(v) for v in gpu_runs.values()]
    ob, gb = float(oracle_runs["base"]), float(gpu_runs["base"])
    so = max(og) / min(og) - 1.0
    sg = max(gg) / min(gg) - 1.0
    err = abs(gb - ob) / ob
    if so <= rtol and sg <= rtol:
        assert err <= rtol, (what, gb, ob, err, so, sg)
        return "bound", err, so, sg
    lo, hi = max(min(og), min(gg)), min(max(og), max(gg))
    assert lo <= hi * (1.0 + rtol) ** 2, (what, "ranges do not overlap", (min(gg), max(gg)), (min(og), max(og)))
    return "ranges overlap", err, so, sg


def check_final_expl(e_g, runs, what, rtol=EXPL_RTOL):
    """Final exploitability of the GPU against the FP64 oracle's runs on the
    same game (`base`) and on summation-order reorderings of it.  Where the
    oracle's own spread is within rtol, the bound is |e_g - e_base| <= rtol
    e_base; where the oracle itself spreads wider (its trajectory depends on
    rounding, Appendix D), e_g must lie inside the oracle's range widened by
    rtol on each side.  Returns (kind, relative error against base, spread)."""
    vals = [float(v) for v in runs.values()]
    base = float(runs["base"])
    lo, hi = min(vals), max(vals)
    spread = hi / lo - 1.0 if lo > 0 else float("inf")
    err = abs(e_g - base) / base if base > 0 else abs(e_g)
    if spread <= rtol:
        assert err <= rtol, (what, e_g, base, err)
        return "bound", err, spread
    assert lo / (1.0 + rtol) <= e_g <= hi * (1.0 + rtol), (what, e_g, lo, hi, spread)
    return "oracle range", err, spread


def oracle_values(o, init, b1_next, alternating):
    """The oracle's counterfactual values V (per sequence) and ev (per
    infoset) of each player's bottom-up pass in the iteration just run, from
    the state before it (init[p] = (r, b)) and, for player 2 under alternating
    updates, player 1's next strategy as the GPU computed it (so a
    regret-matching tie in player 1 cannot leak into player 2's check)."""
    (r1, b1), (r2, b2) = init[1], init[2]
    u1 = o.utility(1, o.sequence_form(2, b2))
    _, V1, ev1 = o.observe_utility(1, u1, b1, r1)
    x1 = o.sequence_form(1, b1_next if alternating else b1)
    _, V2, ev2 = o.observe_utility(2, o.utility(2, x1), b2, r2)
    return {1: (V1[1:], ev1), 2: (V2[1:], ev2)}


def regret_scale(o, p, r_old, r_new, V, ev):
    """Per-sequence magnitude of the regret update r + (V - ev) followed by
    the post-op (a clip or a factor <= 1): an FP32 evaluation of it is off by
    a few ulp of |r_old| + |V| + |ev|, so that (or the vector's RMS, if
    larger) is the scale of the element-wise check."""
    _, na = o.infosets(p)
    ev_seq = np.repeat(ev, na)
    s = np.abs(r_old) + np.abs(V) + np.abs(ev_seq)
    return np.maximum(s, np.sqrt(np.mean(r_new * r_new)))


def random_state(o, p, rng, scale=1.0, t=5):
    """Seeded state for player p of an oracle game: regrets, a behavioural
    strategy on each infoset's simplex, positive average sums."""
    S = o.S[p]
    r = rng.standard_normal(S) * scale
    r[rng.uniform(size=S) < 0.2] = 0.0
    ps, na = o.infosets(p)
    b = np.zeros(S)
    off = 0
    for n in na:
        w = rng.uniform(0.05, 1.0, n)
        b[off:off + n] = w / w.sum()
        off += n
    xbar = np.abs(rng.standard_normal(S + 1)) * 3.0
    return r, b, xbar, t


def strategy_mismatch_ok(b_gpu, b_orc, r_orc_next, na, tol=1e-5, tie=1e-6):
    """Compare next strategies infoset by infoset.  Where the oracle's
    positive-regret sum is at the level of rounding noise, regret matching's
    zero test may legitimately go either way (uniform vs. a vertex), so only
    validity is checked there.  Returns the number of mismatching infosets."""
    off = 0
    scale = max(1.0, np.abs(r_orc_next).max())
    bad = 0
    for n in na:
        sl = slice(off, off + n)
        pos = np.maximum(r_orc_next[sl], 0).sum()
        if pos > tie * scale:
            bad += int(np.abs(b_gpu[sl] - b_orc[sl]).max() > tol)
        else:
            assert abs(b_gpu[sl].sum() - 1.0) < 1e-5 and (b_gpu[sl] >= 0).all()
        off += n
    return bad


def reorder(tree, seed):
    """The same game with its nodes renumbered and each player's infoset ids
    permuted (seeded).  Nodes get a breadth-first numbering in which the
    children of every node come in a random order, so parents still precede
    children; edge labels, chance probabilities and payoffs move with their
    nodes.  Only the order in which the FP64 oracle adds terminals into the
    payoff products and child infosets into counterfactual values changes:
    runs on reordered copies measure the oracle's own summation-order spread."""
    from paper_2605_14277_b300 import games as G
    rng = np.random.default_rng(seed)
    n = tree.n_nodes
    parent = tree.parent.astype(np.int64)
    depth = np.zeros(n, np.int64)
    for _ in range(n):   # parents precede children: converges in (max depth + 1) passes
        nd = depth.copy()
        nd[1:] = depth[parent[1:]] + 1
        if np.array_equal(nd, depth):
            break
        depth = nd
    new = np.full(n, -1, np.int64)
    new[0] = 0
    nxt = 1
    for d in range(1, int(depth.max()) + 1):
        idx = np.nonzero(depth == d)[0]
        order = idx[np.lexsort((rng.random(idx.shape[0]), new[parent[idx]]))]
        new[order] = np.arange(nxt, nxt + order.shape[0])
        nxt += order.shape[0]
    inv = np.empty(n, np.int64)
    inv[new] = np.arange(n)
    par = np.where(parent[inv] < 0, -1, new[np.maximum(parent[inv], 0)])
    kind = tree.kind[inv]
    inf = tree.infoset[inv].copy()
    for p in (1, 2):
        m = kind == p
        if m.any():
            inf[m] = rng.permutation(int(inf[m].max()) + 1)[inf[m]]
    return G.Tree(par, kind, inf, tree.action[inv], tree.chance_prob[inv], tree.payoff[inv],
                  name=tree.name, meta=dict(tree.meta))
