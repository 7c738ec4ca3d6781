"""Host game compiler: layout invariants and an FP64 replay of the kernels'
schedule (units bottom-up in queue order, each unit deepest level first; then
every unit top-down in queue order) over the compiled index arrays, checked
against the oracle.  CPU only."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2605_14277_b300 import games as G
from tests.layout_probe import Layout, down_bytes, span16, up_bytes, work16
from tests.refimpl import SeqForm


def small_set():
    return [G.small_random_game(1), G.poker_game(), G.rps(),
            G.random_game(5, depth=5, chance={0: 3, 3: 2}, actions=(2, 3), payoff="normal"),
            G.matrix_game(G.random_2x2_no_saddle(1))]


def check_invariants(lay, G_):
    for p in (0, 1):
        d = lay.pl[p]
        inf_seq, seq_child, inf_par = d["inf_seq"], d["seq_child"], d["inf_par"]
        J, S = inf_seq.shape[0] - 1, seq_child.shape[0] - 1
        assert inf_seq[0] == 0 and inf_seq[-1] == S and (np.diff(inf_seq) >= 1).all()
        assert seq_child[0] == G_ and seq_child[-1] == J and (np.diff(seq_child) >= 0).all()
        assert (inf_par[:G_] == -1).all()
        for j in range(G_, J):
            q = inf_par[j]
            assert seq_child[q] <= j < seq_child[q + 1]
        # every infoset covered exactly once by the units
        cover = np.zeros(J, np.int64)
        rng = d["ranges"]
        units = d["units"]
        unit_of = {}
        for ui, (g, lvl0, nlvl, r0, flags, par, nch, depth) in enumerate(units):
            assert nlvl >= 1
            prev = None
            for k in range(nlvl):
                lo, hi, s0, s1, n0, n1 = rng[r0 + 6 * k: r0 + 6 * k + 6]
                assert hi > lo
                assert s0 == inf_seq[lo] and s1 == inf_seq[hi]
                assert n0 == d["m_ptr"][s0] and n1 == d["m_ptr"][s1]
                cover[lo:hi] += 1
                for j in range(lo, hi):
                    unit_of[j] = (ui, k)
                if prev is not None:
                    # level k holds exactly the children of level k-1
                    assert lo == seq_child[inf_seq[prev[0]]] and hi == seq_child[inf_seq[prev[1]]]
                prev = (lo, hi)
        assert (cover == 1).all()
        # tree structure: a unit's top level hangs below its parent's deepest
        # level; roots are level 0; child counts and depths agree
        nchild = np.zeros(len(units), np.int64)
        for ui, (g, lvl0, nlvl, r0, flags, par, nch, depth) in enumerate(units):
            lo, hi = rng[r0], rng[r0 + 1]
            if par < 0:
                assert lvl0 == 0 and depth == 0 and d["game_root"][g] == ui and hi - lo == 1
                continue
            nchild[par] += 1
            pg, plvl0, pnlvl = units[par][0], units[par][1], units[par][2]
            assert pg == g and plvl0 + pnlvl == lvl0 and units[par][7] + 1 == depth
            assert units[par][4] & 2
            for j in range(lo, hi):
                pinf = np.searchsorted(inf_seq, inf_par[j], side="right") - 1
                assert unit_of[pinf] == (par, pnlvl - 1)
        assert nchild.tolist() == units[:, 6].tolist()
        # internal units have children; their deepest level's children are
        # exactly the children units' top levels, and that range follows the
        # unit's levels as one more record
        for ui, (g, lvl0, nlvl, r0, flags, par, nch, depth) in enumerate(units):
            lo, hi = rng[r0 + 6 * (nlvl - 1)], rng[r0 + 6 * (nlvl - 1) + 1]
            c0, c1 = seq_child[inf_seq[lo]], seq_child[inf_seq[hi]]
            assert bool(flags & 2) == (nch > 0) == (c1 > c0)
            if flags & 2:
                assert rng[r0 + 6 * nlvl: r0 + 6 * nlvl + 6].tolist() == [c0, c1, 0, 0, 0, 0]
                kids = [v for v in range(len(units)) if units[v][5] == ui]
                assert min(rng[units[v][3]] for v in kids) == c0
                assert max(rng[units[v][3] + 1] for v in kids) == c1
            # below-the-root flag
            assert bool(flags & 4) == (par >= 0 and units[par][5] < 0)
        # queues: leaves for the bottom-up pass; all units, parents first, for
        # the top-down pass
        # the bottom-up queue holds every unit, each after all its children
        assert sorted(d["up_queue"].tolist()) == list(range(len(units)))
        upos = np.empty(len(units), np.int64)
        upos[d["up_queue"]] = np.arange(len(units))
        for ui in range(len(units)):
            if units[ui][5] >= 0:
                assert upos[units[ui][5]] > upos[ui]
        # top-down units: merged runs of siblings; they cover every infoset
        # once, hang below their parent's deepest level, and come after it
        # each starts with its ancestor chain (flags >> 16 records, the game's
        # root level first): every chain level holds exactly the infosets
        # that own the parents of the level below it
        du = d["dunits"]
        cover = np.zeros(J, np.int64)
        dunit_of = {}

        def owner(seq):
            return np.searchsorted(inf_seq, seq, side="right") - 1

        for di, (g, lvl0, nlvl, r0, flags, par, nch, depth) in enumerate(du):
            n_anc = flags >> 16
            assert n_anc == lvl0 and nlvl > n_anc
            recs = [rng[r0 + 6 * k: r0 + 6 * k + 4] for k in range(nlvl)]
            for k, (lo, hi, s0, s1) in enumerate(recs):
                assert hi > lo and s0 == inf_seq[lo] and s1 == inf_seq[hi]
                if k == 0:
                    assert (inf_par[lo:hi] < 0).all() and hi - lo == 1 and d["seq_game"][s0] == g
                else:
                    plo, phi = recs[k - 1][0], recs[k - 1][1]
                    if k <= n_anc:   # a chain level, or the unit's top level: parents in the level above
                        assert plo == owner(inf_par[lo]) and phi == owner(inf_par[hi - 1]) + 1
                    if k > n_anc:    # own levels: the children of the level above
                        assert lo == seq_child[inf_seq[plo]] and hi == seq_child[inf_seq[phi]]
                if k >= n_anc:
                    cover[lo:hi] += 1
                    for j in range(lo, hi):
                        dunit_of[j] = (di, k)
        assert (cover == 1).all()
        nchild_d = np.zeros(len(du), np.int64)
        for di, (g, lvl0, nlvl, r0, flags, par, nch, depth) in enumerate(du):
            n_anc = flags >> 16
            lo, hi = rng[r0 + 6 * n_anc], rng[r0 + 6 * n_anc + 1]
            if par < 0:
                assert lvl0 == 0 and hi - lo == 1
                continue
            nchild_d[par] += 1
            for j in range(lo, hi):
                pinf = owner(inf_par[j])
                assert dunit_of[pinf] == (par, du[par][2] - 1)
            assert bool(flags & 4) == (du[par][5] < 0)
        assert nchild_d.tolist() == du[:, 6].tolist()
        assert len(du) <= len(units)
        assert sorted(d["down_queue"].tolist()) == list(range(len(du)))
        pos = np.empty(len(du), np.int64)
        pos[d["down_queue"]] = np.arange(len(du))
        for di in range(len(du)):
            if du[di][5] >= 0:
                assert pos[du[di][5]] < pos[di]
        assert (np.diff(du[d["down_queue"], 7]) >= 0).all()


@pytest.mark.parametrize("item_bytes", [0, 600, 4000])
def test_layout_invariants_single_and_batch(item_bytes):
    trees = small_set()
    for t in trees:
        check_invariants(Layout([t], item_bytes=item_bytes), 1)
    check_invariants(Layout(trees, item_bytes=item_bytes), len(trees))


def test_staged_units_fit_their_buffer():
    """every unit flagged as staged fits the shared-memory buffer (both passes)"""
    for item_bytes in (2000, 8000, 96 * 1024):
        lay = Layout([G.poker_game(), G.random_game(5, depth=5, chance={0: 3, 3: 2}, actions=(2, 3),
                                                    payoff="normal")], item_bytes=item_bytes)
        for p in (0, 1):
            d = lay.pl[p]
            n_staged = 0
            for (g, lvl0, nlvl, r0, flags, par, nch, depth) in d["dunits"]:
                # own levels and the ancestor chain staged with them
                rng = d["ranges"][r0: r0 + 6 * nlvl].reshape(-1, 6)
                fd = sum(down_bytes(s1 - s0, j1 - j0) for j0, j1, s0, s1, n0, n1 in rng)
                if flags & 1:
                    assert fd <= item_bytes and nlvl <= 24
            for (g, lvl0, nlvl, r0, flags, par, nch, depth) in d["units"]:
                rng = d["ranges"][r0: r0 + 6 * nlvl].reshape(-1, 6)
                fu = sum(up_bytes(s1 - s0, j1 - j0, n1 - n0) for j0, j1, s0, s1, n0, n1 in rng)
                fd = sum(down_bytes(s1 - s0, j1 - j0) for j0, j1, s0, s1, n0, n1 in rng)
                if flags & 2:
                    c0, c1 = d["ranges"][r0 + 6 * nlvl: r0 + 6 * nlvl + 2]
                    fu += 16 * ((4 * (c1 - c0) + 32 + 15) // 16)
                if flags & 1:
                    n_staged += 1
                    assert fu <= item_bytes and fd <= item_bytes and nlvl <= 24
            assert n_staged > 0


def test_deep_games_get_several_tiers():
    """a game far larger than one unit is cut into a tree several tiers deep,
    with every unit staged"""
    t = G.random_game(11, depth=9, chance={0: 4, 4: 3}, actions=(3, 4), payoff="normal")
    lay = Layout([t], item_bytes=3000)
    for p in (0, 1):
        d = lay.pl[p]
        assert d["game_tiers"][0] >= 3
        assert d["units"][:, 7].max() + 1 == d["game_tiers"][0]
        assert (d["units"][:, 4] & 1).all()


def test_payoff_matrix_matches_sequence_form():
    trees = small_set()
    lay = Layout(trees, item_bytes=3000)
    d1, d2 = lay.pl[0], lay.pl[1]
    S1, S2 = d1["m_ptr"].shape[0] - 1, d2["m_ptr"].shape[0] - 1
    M = np.zeros((S1, S2))
    for r in range(S1):
        for k in range(d1["m_ptr"][r], d1["m_ptr"][r + 1]):
            M[r, d1["m_col"][k]] += d1["m_val64"][k]
    MT = np.zeros((S2, S1))
    for r in range(S2):
        for k in range(d2["m_ptr"][r], d2["m_ptr"][r + 1]):
            MT[r, d2["m_col"][k]] += d2["m_val64"][k]
    assert np.array_equal(M, MT.T)
    for g, t in enumerate(trees):
        sf = SeqForm(t)
        f1 = np.concatenate([[g], lay.caller_to_forest(0, g)])
        f2 = np.concatenate([[g], lay.caller_to_forest(1, g)])
        assert np.allclose(M[np.ix_(f1, f2)], sf.M, rtol=1e-15, atol=1e-15)
        # no payoff between games
        assert np.abs(M[np.ix_(f1, np.setdiff1d(np.arange(S2), f2))]).max(initial=0) == 0


# ---------------------------------------------------------------- schedule replay

class Sim:
    """FP64 replay of the kernel schedule on the compiled layout."""

    def __init__(self, lay, G_):
        self.lay, self.G = lay, G_

    def rows(self, p, xo, sign):
        d = self.lay.pl[p]
        ptr, col, val = d["m_ptr"], d["m_col"], d["m_val64"]
        u = np.zeros(ptr.shape[0] - 1)
        for r in range(u.shape[0]):
            u[r] = sign * np.dot(val[ptr[r]:ptr[r + 1]], xo[col[ptr[r]:ptr[r + 1]]])
        return u

    def up(self, p, st, xo, sign, variant, t, alpha, beta):
        d = self.lay.pl[p]
        inf_seq, seq_child, rng = d["inf_seq"], d["seq_child"], d["ranges"]
        u = self.rows(p, xo, sign)
        ev = np.full(inf_seq.shape[0] - 1, np.nan)
        r, b = st[p]["r"], st[p]["b"]

        def step(j, tg):
            s0, s1 = inf_seq[j], inf_seq[j + 1]
            V = np.array([u[s] + ev[seq_child[s]:seq_child[s + 1]].sum() for s in range(s0, s1)])
            assert not np.isnan(V).any()
            e = float(b[s0:s1] @ V)
            ev[j] = e
            rn = r[s0:s1] + (V - e)
            if variant in (1, 3):
                rn = np.maximum(rn, 0.0)
            elif variant == 2:
                fp = tg ** alpha / (tg ** alpha + 1)
                fn = tg ** beta / (tg ** beta + 1)
                rn = np.where(rn > 0, rn * fp, np.where(rn < 0, rn * fn, rn))
            r[s0:s1] = rn
            q = rn + (V - e) if variant == 3 else rn
            q = np.maximum(q, 0)
            b[s0:s1] = q / q.sum() if q.sum() > 0 else 1.0 / (s1 - s0)

        units = d["units"]

        def run(ui):
            g, lvl0, nlvl, r0 = units[ui][:4]
            for k in range(nlvl - 1, -1, -1):
                for j in range(rng[r0 + 6 * k], rng[r0 + 6 * k + 1]):
                    step(j, t[g])

        # queue order; an internal unit runs once all its children are done
        done = np.zeros(len(units), np.int64)
        for ui in d["up_queue"]:
            assert done[ui] == units[ui][6]
            run(ui)
            if units[ui][5] >= 0:
                done[units[ui][5]] += 1

    def down(self, p, st, w):
        d = self.lay.pl[p]
        inf_seq, rng, inf_par = d["inf_seq"], d["ranges"], d["inf_par"]
        x, xbar, b = st[p]["x"], st[p]["xbar"], st[p]["b"]
        units = d["dunits"]
        # every unit works from its own values only: the next x of its
        # ancestor chain (recomputed, not written) and of its own levels
        for ui in d["down_queue"]:
            g, lvl0, nlvl, r0, flags, par = units[ui][:6]
            n_anc = flags >> 16
            local = {}
            for k in range(nlvl):
                for j in range(rng[r0 + 6 * k], rng[r0 + 6 * k + 1]):
                    xp = 1.0 if inf_par[j] < 0 else local[inf_par[j]]
                    for s in range(inf_seq[j], inf_seq[j + 1]):
                        local[s] = xp * b[s]
                        if k >= n_anc:
                            xbar[s] += w[g] * x[s]
                            x[s] = local[s]

    def iteration(self, st, variant, alpha, beta, gamma, alternating, t_done):
        t = t_done + 1.0
        w = t ** gamma
        if alternating:
            self.up(0, st, st[1]["x"], 1.0, variant, t, alpha, beta)
            self.down(0, st, w)
            self.up(1, st, st[0]["x"], -1.0, variant, t, alpha, beta)
            self.down(1, st, w)
        else:
            self.up(0, st, st[1]["x"], 1.0, variant, t, alpha, beta)
            self.up(1, st, st[0]["x"], -1.0, variant, t, alpha, beta)
            self.down(0, st, w)
            self.down(1, st, w)


@pytest.mark.parametrize("variant,alt", [(0, False), (1, True), (2, True), (3, True), (2, False)])
def test_schedule_matches_oracle_one_iteration(variant, alt):
    trees = [G.random_game(5, depth=5, chance={0: 3, 3: 2}, actions=(2, 3), payoff="normal"),
             G.poker_game(), G.rps()]
    lay = Layout(trees, item_bytes=5000)
    rng = np.random.default_rng(7)
    alpha, beta, gamma = 1.5, 0.0, 2.0
    t0 = 4
    st = {0: {}, 1: {}}
    oracles = []
    for p in (0, 1):
        S = lay.pl[p]["inf_seq"][-1]
        st[p] = {"r": np.zeros(S), "b": np.ones(S), "x": np.zeros(S), "xbar": np.zeros(S)}
    for g, t in enumerate(trees):
        o = Oracle(t)
        for p in (0, 1):
            f = lay.caller_to_forest(p, g)
            r = rng.standard_normal(o.S[p + 1])
            b = o.regret_matching(p + 1, r)
            xb = np.abs(rng.standard_normal(o.S[p + 1] + 1))
            o.set_state(p + 1, r, b, xb, t0)
            st[p]["r"][f] = r
            st[p]["b"][f] = b
            st[p]["xbar"][f] = xb[1:]
            st[p]["xbar"][g] = xb[0]
            x = o.sequence_form(p + 1, b)
            st[p]["x"][f] = x[1:]
            st[p]["x"][g] = 1.0
        o.iterate(1, variant, alpha=alpha, beta=beta, gamma=gamma, alternating=alt)
        oracles.append(o)
    Sim(lay, len(trees)).iteration(st, variant, alpha, beta, gamma, alt, np.full(len(trees), float(t0)))
    for g, o in enumerate(oracles):
        for p in (0, 1):
            f = lay.caller_to_forest(p, g)
            os_ = o.get_state(p + 1)
            assert np.allclose(st[p]["r"][f], os_["r"], rtol=1e-12, atol=1e-12)
            assert np.allclose(st[p]["b"][f], os_["b"], rtol=1e-12, atol=1e-12)
            assert np.allclose(st[p]["xbar"][f], os_["xbar"][1:], rtol=1e-12, atol=1e-12)
            assert abs(st[p]["xbar"][g] - os_["xbar"][0]) < 1e-12


def check_windows(lay):
    """x windows: for every windowed level, the windows are ordered, disjoint,
    more than the gap apart, few, no larger than per-entry gathers, and each
    entry's local column points at its own column once the windows are laid
    out one after another (each at its 16-byte-aligned offset)"""
    n_win = n_all = 0
    for p in (0, 1):
        d = lay.pl[p]
        rng, rwin, win, lcol, col = d["ranges"], d["rwin"], d["win"], d["lcol"], d["m_col"]
        assert rwin.shape[0] == 4 * (rng.shape[0] // 6) and lcol.shape == col.shape
        win = win.reshape(-1, 4)
        windowed = np.zeros(col.shape[0], bool)
        for (g, lvl0, nlvl, r0, flags, par, nch, depth) in d["units"]:
            if flags & 1:
                # the unit's windows are one contiguous run, level by level
                recs = [r0 // 6 + k for k in range(nlvl)]
                for a, b in zip(recs[:-1], recs[1:]):
                    assert rwin[4 * a + 1] == rwin[4 * b]
            for k in range(nlvl):
                rec = r0 // 6 + k
                w0, w1, xb = rwin[4 * rec: 4 * rec + 3]
                n0, n1 = rng[r0 + 6 * k + 4], rng[r0 + 6 * k + 5]
                n_all += n1 - n0
                if w0 == w1:
                    assert xb == (work16(n1 - n0, 4) if flags & 1 else 0)
                    continue
                assert flags & 1, "only staged units carry windows"
                n_win += n1 - n0
                W = win[w0:w1]
                assert len(W) <= 32 and (W[:, 1] > W[:, 0]).all() and (W[:, 3] == k).all()
                assert (W[1:, 0] - W[:-1, 1] >= 16).all()
                sizes = [span16(c1 - c0, 4) for c0, c1 in W[:, :2]]
                assert sum(sizes) == xb <= work16(n1 - n0, 4)
                assert (W[:, 2] == np.concatenate([[0], np.cumsum(sizes)[:-1]])).all()
                smem = np.full(xb // 4, -1, np.int64)
                for c0, c1, off, _ in W:
                    smem[off // 4 + (c0 & 3): off // 4 + (c0 & 3) + (c1 - c0)] = np.arange(c0, c1)
                assert (smem[lcol[n0:n1]] == col[n0:n1]).all()
                windowed[n0:n1] = True
        assert (lcol[~windowed] == col[~windowed]).all()
    return n_win, n_all


def test_x_windows():
    t = G.random_game(11, depth=9, chance={0: 4, 4: 3}, actions=(3, 4), payoff="normal")
    n_win, n_all = check_windows(Layout([t], item_bytes=48 * 1024))
    assert n_win >= 0.4 * n_all
    for trees in (small_set(), [G.poker_game()]):
        check_windows(Layout(trees, item_bytes=48 * 1024))


def test_top_down_units_fit_one_round_of_ctas(monkeypatch):
    """The top-down pass's units are independent, so the packer merges them to
    the smallest footprint that leaves no more units than CTAs resident at
    once: the large game's top-down pass is then one round (296 CTAs), while
    each unit still fits its buffer."""
    monkeypatch.setenv("LAYOUT_PROBE_SLOTS", "296")
    lay = Layout([G.large_random_game(3)], item_bytes=48 * 1024)
    for p in (0, 1):
        d = lay.pl[p]
        du = d["dunits"]
        assert len(du) <= 296
        # not merged further than needed: at least half the CTAs get a unit
        assert len(du) >= 148
        for (g, lvl0, nlvl, r0, flags, par, nch, depth) in du:
            rng = d["ranges"][r0: r0 + 6 * nlvl].reshape(-1, 6)
            fd = sum(down_bytes(s1 - s0, j1 - j0) for j0, j1, s0, s1, n0, n1 in rng)
            assert (flags & 1) == 0 or fd <= 48 * 1024
