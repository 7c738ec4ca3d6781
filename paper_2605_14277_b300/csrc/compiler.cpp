// Host game compiler: flat game trees -> level-sorted CSR/segment layout.
//
// Builds, per player, the tree-form sequential decision process of each game
// (decision points = infosets, sequences (j, a), parent sequence p_j; Sec. 2.1),
// the payoff matrix M[s1, s2] = sum over terminals z with those sequences of
// chance reach * u1(z) (two-player utilities as one sparse product, Sec. 2.1),
// and the breadth-first forest numbering described in layout.h.  The logic
// matrices A, B, C and the level graphs L^(d) of Sec. 3.1-3.2 are not stored
// as matrices: each has at most one nonzero per column, so each becomes an
// index array (inf_seq, seq_child, inf_par) over the breadth-first order.
// Finally each player's levels are cut into a tree of units that each fit
// one shared-memory buffer of the CUDA passes.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "layout.h"

namespace cfrb {

namespace {

enum { K_CHANCE = 0, K_P1 = 1, K_P2 = 2, K_TERM = 3 };

struct PlayerSF {
    int32_t J = 0, S = 0;
    std::vector<int32_t> nact, off, par;    // per caller infoset; par = caller seq, -1 = empty
    std::vector<int32_t> kid_ptr, kid_inf;  // child infosets of caller seq s at kid_ptr[s+1]..; [0] = empty
};

struct GameSF {
    PlayerSF p[2];
    std::vector<int32_t> ts1, ts2;          // caller seq of each terminal, -1 = empty
    std::vector<double> tw;                 // chance reach * payoff
    double range = 0.0;
    int64_t nodes = 0;
};

bool fail(std::string *err, const std::string &m) {
    if (err) *err = m;
    return false;
}

bool compile_game(const TreeView &t, GameSF *g, std::string *err) {
    const int64_t n = t.n_nodes;
    g->nodes = n;
    if (n < 1) return fail(err, "empty tree");
    if (t.parent[0] != -1) return fail(err, "node 0 must be the root (parent -1)");
    // pass 1: node kinds, parents, child counts, infoset ids per player, terminals
    std::vector<int32_t> nch(n, 0);
    int64_t Jp[2] = {0, 0}, nterm = 0;
    for (int64_t i = 0; i < n; i++) {
        const int k = t.kind[i];
        if (k < 0 || k > 3) return fail(err, "bad node kind at " + std::to_string(i));
        if (i > 0) {
            const int64_t q = t.parent[i];
            if (q < 0 || q >= i) return fail(err, "parent must precede child at " + std::to_string(i));
            if (t.kind[q] == K_TERM) return fail(err, "terminal with children at " + std::to_string(q));
            nch[q]++;
        }
        if (k == K_P1 || k == K_P2) {
            if (t.infoset[i] < 0) return fail(err, "decision node without infoset at " + std::to_string(i));
            Jp[k - 1] = std::max<int64_t>(Jp[k - 1], (int64_t)t.infoset[i] + 1);
        } else if (k == K_TERM) {
            if (!std::isfinite(t.payoff[i])) return fail(err, "non-finite payoff at " + std::to_string(i));
            nterm++;
        }
    }
    for (int p = 0; p < 2; p++) {
        if (Jp[p] > INT32_MAX / 2) return fail(err, "too many infosets");
        g->p[p].J = (int32_t)Jp[p];
        g->p[p].nact.assign(Jp[p], 0);
        g->p[p].par.assign(Jp[p], INT32_MIN);
    }
    // pass 2: every non-terminal has children; each infoset's action count;
    // the start of each node's action-label slots
    std::vector<int32_t> coff(n + 1, 0);
    for (int64_t i = 0; i < n; i++) {
        const int k = t.kind[i];
        if (k != K_TERM && nch[i] == 0) return fail(err, "non-terminal without children at " + std::to_string(i));
        if (k == K_P1 || k == K_P2) {
            int32_t &na = g->p[k - 1].nact[t.infoset[i]];
            if (na == 0) na = nch[i];
            else if (na != nch[i]) return fail(err, "infoset action-count mismatch");
        }
        if (coff[i] > INT32_MAX - nch[i]) return fail(err, "too many nodes");
        coff[i + 1] = coff[i] + nch[i];
    }
    // caller sequence numbering
    for (int p = 0; p < 2; p++) {
        PlayerSF &P = g->p[p];
        P.off.assign(P.J, 0);
        int64_t s = 0;
        for (int64_t j = 0; j < P.J; j++) {
            if (P.nact[j] == 0) return fail(err, "infoset ids are not dense");
            P.off[j] = (int32_t)s;
            s += P.nact[j];
        }
        if (s > INT32_MAX / 2) return fail(err, "too many sequences");
        P.S = (int32_t)s;
    }
    // pass 3, top-down (parents precede children): action labels 0..nch-1 once
    // each; chance probabilities valid (their sums checked once a node's last
    // child is seen, in the running sum kept per chance node); each node's own
    // sequence per player and chance reach; perfect recall (all nodes of an
    // infoset share its parent sequence); terminals
    std::vector<uint8_t> seen(n > 1 ? n - 1 : 1, 0);
    std::vector<int32_t> seq1(n, -1), seq2(n, -1);
    std::vector<double> reach(n, 1.0);   // the chance reach, and for a chance node the running sum of its
    std::vector<double> psum;            // children's probabilities (psum, indexed by chance node rank)
    std::vector<int32_t> crank;
    {
        int64_t nc = 0;
        for (int64_t i = 0; i < n; i++) nc += t.kind[i] == K_CHANCE;
        if (nc > 0) {
            crank.assign(n, -1);
            psum.assign(nc, 0.0);
            nc = 0;
            for (int64_t i = 0; i < n; i++)
                if (t.kind[i] == K_CHANCE) crank[i] = (int32_t)nc++;
        }
    }
    g->ts1.reserve(nterm);
    g->ts2.reserve(nterm);
    g->tw.reserve(nterm);
    double mn = INFINITY, mx = -INFINITY;
    auto own_infoset = [&](int64_t i) {
        const int k = t.kind[i];
        if (k != K_P1 && k != K_P2) return true;
        PlayerSF &P = g->p[k - 1];
        const int32_t own = (k == K_P1) ? seq1[i] : seq2[i];
        int32_t &pj = P.par[t.infoset[i]];
        if (pj == INT32_MIN) pj = own;
        else if (pj != own)
            return fail(err, "imperfect recall: infoset " + std::to_string(t.infoset[i]) + " of player " +
                                 std::to_string(k) + " has two parent sequences");
        return true;
    };
    if (!own_infoset(0)) return false;
    if (t.kind[0] == K_TERM) {
        g->ts1.push_back(-1);
        g->ts2.push_back(-1);
        g->tw.push_back(t.payoff[0]);
        mn = mx = t.payoff[0];
    }
    for (int64_t i = 1; i < n; i++) {
        const int64_t q = t.parent[i];
        const int kq = t.kind[q];
        const int32_t a = t.action[i];
        if (a < 0 || a >= nch[q]) return fail(err, "action label out of range at " + std::to_string(i));
        if (seen[coff[q] + a]) return fail(err, "duplicate action label below " + std::to_string(q));
        seen[coff[q] + a] = 1;
        double rq = reach[q];
        if (kq == K_CHANCE) {
            const double pr = t.chance_prob[i];
            if (!(pr >= 0.0 && pr <= 1.0)) return fail(err, "bad chance probability at " + std::to_string(i));
            psum[crank[q]] += pr;
            rq *= pr;
        }
        reach[i] = rq;
        seq1[i] = (kq == K_P1) ? g->p[0].off[t.infoset[q]] + a : seq1[q];
        seq2[i] = (kq == K_P2) ? g->p[1].off[t.infoset[q]] + a : seq2[q];
        if (!own_infoset(i)) return false;
        if (t.kind[i] == K_TERM) {
            g->ts1.push_back(seq1[i]);
            g->ts2.push_back(seq2[i]);
            g->tw.push_back(reach[i] * t.payoff[i]);
            mn = std::min(mn, t.payoff[i]);
            mx = std::max(mx, t.payoff[i]);
        }
    }
    for (int64_t i = 0; i < n; i++)
        if (t.kind[i] == K_CHANCE && std::fabs(psum[crank[i]] - 1.0) > 1e-9)
            return fail(err, "chance probabilities do not sum to 1 at " + std::to_string(i));
    // children of each caller sequence (index 0 = empty sequence), sorted by
    // infoset id; a cycle leaves infosets unreachable, which the forest
    // numbering detects
    for (int p = 0; p < 2; p++) {
        PlayerSF &P = g->p[p];
        P.kid_ptr.assign((size_t)P.S + 2, 0);
        for (int32_t j = 0; j < P.J; j++) P.kid_ptr[P.par[j] + 2]++;
        for (int64_t s = 1; s < (int64_t)P.S + 2; s++) P.kid_ptr[s] += P.kid_ptr[s - 1];
        P.kid_inf.assign(P.J, 0);
        std::vector<int32_t> fill(P.kid_ptr.begin(), P.kid_ptr.end() - 1);
        for (int32_t j = 0; j < P.J; j++) P.kid_inf[fill[P.par[j] + 1]++] = j;
    }
    g->range = g->ts1.empty() ? 0.0 : mx - mn;
    return true;
}

template <class F>
void parallel_for(int64_t n, F f) {
    unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 32u));
    if (n < 4 || nt == 1) {
        for (int64_t i = 0; i < n; i++) f(i);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> th;
    for (unsigned k = 0; k < nt; k++)
        th.emplace_back([&]() {
            for (int64_t i; (i = next.fetch_add(1)) < n;) f(i);
        });
    for (auto &x : th) x.join();
}

}  // namespace

int compile_forest(const TreeView *games, int64_t G, const CompileOptions &opt, Layout *out, std::string *err) {
    if (G < 1) {
        if (err) *err = "no games";
        return ST_INVALID;
    }
    std::vector<GameSF> gs(G);
    std::vector<std::string> errs(G);
    std::vector<char> ok(G, 0);
    parallel_for(G, [&](int64_t g) { ok[g] = compile_game(games[g], &gs[g], &errs[g]); });
    for (int64_t g = 0; g < G; g++)
        if (!ok[g]) {
            if (err) *err = "game " + std::to_string(g) + ": " + errs[g];
            return ST_INVALID;
        }
    Layout &L = *out;
    L.G = G;
    L.game_nodes.resize(G);
    L.game_range.resize(G);
    for (int64_t g = 0; g < G; g++) {
        L.game_nodes[g] = gs[g].nodes;
        L.game_range[g] = gs[g].range;
    }
    // caller seq -> forest seq, per game and player
    std::vector<std::vector<int32_t>> gseq[2];
    // per player, per game, per level: infoset range
    std::vector<std::vector<std::pair<int32_t, int32_t>>> glvs[2];
    for (int p = 0; p < 2; p++) {
        PlayerLayout &P = L.pl[p];
        gseq[p].resize(G);
        int64_t S = G, J = G;
        for (int64_t g = 0; g < G; g++) {
            S += gs[g].p[p].S;
            J += gs[g].p[p].J;
            gseq[p][g].assign(gs[g].p[p].S, -1);
        }
        if (S >= INT32_MAX || J >= INT32_MAX) {
            if (err) *err = "forest too large for 32-bit indices";
            return ST_INVALID;
        }
        P.S = S;
        P.J = J;
        P.inf_seq.assign(J + 1, 0);
        P.seq_child.assign(S + 1, 0);
        P.inf_par.assign(J, -1);
        P.seq_game.assign(S, 0);
        P.game_J.resize(G);
        P.game_S.resize(G);
        P.game_jbase.assign(G + 1, 0);
        P.game_sbase.assign(G + 1, 0);
        for (int64_t g = 0; g < G; g++) {
            P.game_J[g] = gs[g].p[p].J;
            P.game_S[g] = gs[g].p[p].S;
            P.game_jbase[g + 1] = P.game_jbase[g] + gs[g].p[p].J;
            P.game_sbase[g + 1] = P.game_sbase[g] + gs[g].p[p].S;
        }
        P.ext_inf.assign(P.game_jbase[G], -1);
        P.ext_seq0.assign(P.game_jbase[G], 0);
        // breadth-first numbering over the forest.  A frontier entry is
        // (game, caller seq or -1, forest seq).
        struct Fr {
            int32_t g, cs, fs;
        };
        std::vector<Fr> cur, nxt;
        int32_t jn = 0, sn = 0;
        std::vector<int32_t> lvl_lo;   // first infoset of each level
        for (int64_t g = 0; g < G; g++) {   // level 0: one root pseudo-infoset per game
            P.inf_seq[jn] = sn;
            P.inf_par[jn] = -1;
            P.seq_game[sn] = (int32_t)g;
            cur.push_back({(int32_t)g, -1, sn});
            jn++;
            sn++;
        }
        lvl_lo.push_back(0);
        while (!cur.empty()) {
            lvl_lo.push_back(jn);   // start of the level created in this pass
            nxt.clear();
            for (const Fr &f : cur) {
                const PlayerSF &Q = gs[f.g].p[p];
                P.seq_child[f.fs] = jn;
                for (int32_t k = Q.kid_ptr[f.cs + 1]; k < Q.kid_ptr[f.cs + 2]; k++) {
                    const int32_t jx = Q.kid_inf[k];
                    P.inf_seq[jn] = sn;
                    P.inf_par[jn] = f.fs;
                    const int64_t e = P.game_jbase[f.g] + jx;
                    P.ext_inf[e] = jn;
                    P.ext_seq0[e] = Q.off[jx];
                    for (int32_t a = 0; a < Q.nact[jx]; a++) {
                        gseq[p][f.g][Q.off[jx] + a] = sn;
                        P.seq_game[sn] = f.g;
                        nxt.push_back({f.g, Q.off[jx] + a, sn});
                        sn++;
                    }
                    P.max_actions = std::max(P.max_actions, Q.nact[jx]);
                    jn++;
                }
            }
            cur.swap(nxt);
        }
        if (jn != J || sn != S) {
            if (err)
                *err = "player " + std::to_string(p + 1) +
                       ": infosets unreachable from the root (cyclic parent sequences)";
            return ST_INVALID;
        }
        P.inf_seq[J] = sn;
        P.seq_child[S] = jn;
        for (int64_t s = 1; s <= S; s++)
            if (P.seq_child[s] < P.seq_child[s - 1]) {
                if (err) *err = "internal: non-monotone child pointers";
                return ST_INVALID;
            }
        // the last pass created an empty level whose start closes the list
        P.n_levels = (int32_t)lvl_lo.size() - 1;
        // per game, per level infoset ranges
        auto &glv = glvs[p];
        glv.assign(G, {});
        for (int32_t d = 0; d < P.n_levels; d++) {
            int32_t j = lvl_lo[d];
            const int32_t e = lvl_lo[d + 1];
            while (j < e) {
                const int32_t g = P.seq_game[P.inf_seq[j]];
                int32_t k = j;
                while (k < e && P.seq_game[P.inf_seq[k]] == g) k++;
                glv[g].push_back({j, k});
                j = k;
            }
        }
    }
    // ---- payoff matrix in forest numbering, CSR by player-1 rows and by player-2 rows
    int64_t Z0 = 0;
    for (int64_t g = 0; g < G; g++) Z0 += (int64_t)gs[g].tw.size();
    if (Z0 >= INT32_MAX) {
        if (err) *err = "too many terminals for 32-bit offsets";
        return ST_INVALID;
    }
    auto fseq = [&](int p, int64_t g, int32_t cs) -> int32_t { return cs < 0 ? (int32_t)g : gseq[p][g][cs]; };
    {
        PlayerLayout &A = L.pl[0];
        std::vector<int32_t> cnt(A.S + 1, 0);
        for (int64_t g = 0; g < G; g++)
            for (size_t z = 0; z < gs[g].tw.size(); z++) cnt[fseq(0, g, gs[g].ts1[z]) + 1]++;
        for (int64_t s = 0; s < A.S; s++) cnt[s + 1] += cnt[s];
        std::vector<int32_t> col(Z0);
        std::vector<double> val(Z0);
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t g = 0; g < G; g++)
            for (size_t z = 0; z < gs[g].tw.size(); z++) {
                const int32_t r = fseq(0, g, gs[g].ts1[z]);
                const int32_t k = fill[r]++;
                col[k] = fseq(1, g, gs[g].ts2[z]);
                val[k] = gs[g].tw[z];
            }
        // merge duplicates within each row (sorted by column, stable: the
        // entries of one column are added in terminal order).  Rows are
        // short, so each is sorted in place by insertion (stable).
        A.m_ptr.assign(A.S + 1, 0);
        A.m_col.clear();
        A.m_val64.clear();
        A.m_col.reserve(Z0);
        A.m_val64.reserve(Z0);
        for (int64_t r = 0; r < A.S; r++) {
            const int32_t k0 = cnt[r], k1 = cnt[r + 1];
            for (int32_t k = k0 + 1; k < k1; k++) {
                const int32_t c = col[k];
                const double v = val[k];
                int32_t m = k;
                for (; m > k0 && col[m - 1] > c; m--) {
                    col[m] = col[m - 1];
                    val[m] = val[m - 1];
                }
                col[m] = c;
                val[m] = v;
            }
            for (int32_t k = k0; k < k1; k++) {
                if ((int64_t)A.m_col.size() > A.m_ptr[r] && A.m_col.back() == col[k])
                    A.m_val64.back() += val[k];
                else {
                    A.m_col.push_back(col[k]);
                    A.m_val64.push_back(val[k]);
                }
            }
            A.m_ptr[r + 1] = (int32_t)A.m_col.size();
        }
        L.Z = (int64_t)A.m_col.size();
        A.m_val.resize(L.Z);
        for (int64_t k = 0; k < L.Z; k++) A.m_val[k] = (float)A.m_val64[k];
        // transpose for player-2 rows
        PlayerLayout &B = L.pl[1];
        B.m_ptr.assign(B.S + 1, 0);
        for (int64_t k = 0; k < L.Z; k++) B.m_ptr[A.m_col[k] + 1]++;
        for (int64_t s = 0; s < B.S; s++) B.m_ptr[s + 1] += B.m_ptr[s];
        B.m_col.resize(L.Z);
        B.m_val64.resize(L.Z);
        B.m_val.resize(L.Z);
        std::vector<int32_t> f2(B.m_ptr.begin(), B.m_ptr.end() - 1);
        for (int64_t r = 0; r < A.S; r++)
            for (int32_t k = A.m_ptr[r]; k < A.m_ptr[r + 1]; k++) {
                const int32_t q = f2[A.m_col[k]]++;
                B.m_col[q] = (int32_t)r;
                B.m_val64[q] = A.m_val64[k];
                B.m_val[q] = A.m_val[k];
            }
    }
    // ---- units: per game and player, a tree of units, each of which fits one
    // shared-memory buffer ----------------------------------------------------
    for (int p = 0; p < 2; p++) {
        PlayerLayout &P = L.pl[p];
        const auto &glv = glvs[p];
        const int64_t J = P.J;
        // own footprint of each infoset (raw bytes, without per-level slack)
        // and the footprint of its whole subtree
        std::vector<int64_t> own(J, 0), raw_up(J, 0);
        for (int64_t j = J - 1; j >= 0; j--) {
            int64_t u = 8 + 8;   // infoset: segment pointer + ev
            int64_t sub = 0;
            for (int32_t q = P.inf_seq[j]; q < P.inf_seq[j + 1]; q++) {
                const int64_t nz = P.m_ptr[q + 1] - P.m_ptr[q];
                u += 24 + 12 * nz;   // r, b, child and row pointers, V; payoff column, value, gathered x
                for (int32_t c = P.seq_child[q]; c < P.seq_child[q + 1]; c++) sub += raw_up[c];
            }
            own[j] = u;
            raw_up[j] = u + sub;
        }
        const int64_t slack_per_level = 8 * 48;
        std::vector<int64_t> f(J, 0);   // subtree footprint truncated at a tier's bottom
        P.units.clear();
        P.ranges.clear();
        P.rwin.clear();
        P.win.clear();
        P.lcol = P.m_col;
        P.game_root.assign(G, -1);
        P.game_tiers.assign(G, 0);
        auto push_level = [&](int32_t j0, int32_t j1) {
            const int32_t s0 = P.inf_seq[j0], s1 = P.inf_seq[j1];
            P.ranges.push_back(j0);
            P.ranges.push_back(j1);
            P.ranges.push_back(s0);
            P.ranges.push_back(s1);
            P.ranges.push_back(P.m_ptr[s0]);
            P.ranges.push_back(P.m_ptr[s1]);
            for (int k = 0; k < 4; k++) P.rwin.push_back(0);
        };
        // x windows of level k of a staged unit (payoff entries [n0, n1)): the
        // sorted distinct columns cut wherever two are more than kWinGap
        // apart.  Taken when at most kMaxWin windows together need no more
        // shared memory than per-entry gathers.
        std::vector<int32_t> cols, wend;
        std::vector<int64_t> wbase;
        std::vector<uint8_t> mark;
        auto windows = [&](int64_t rec, int32_t k, int32_t n0, int32_t n1) {
            const int32_t here = (int32_t)(P.win.size() / 4);
            P.rwin[4 * rec] = P.rwin[4 * rec + 1] = here;
            P.rwin[4 * rec + 2] = (int32_t)work16(n1 - n0, 4);
            if (n1 <= n0) return;
            // the level's distinct columns in order: marked in a table over
            // their span when that span is small (clustered columns), else sorted
            int32_t clo = P.m_col[n0], chi = P.m_col[n0];
            for (int32_t e = n0; e < n1; e++) {
                clo = std::min(clo, P.m_col[e]);
                chi = std::max(chi, P.m_col[e]);
            }
            const int64_t span = (int64_t)chi - clo + 1;
            if (span <= 8 * (int64_t)(n1 - n0) + 4096) {
                mark.assign(span, 0);
                for (int32_t e = n0; e < n1; e++) mark[P.m_col[e] - clo] = 1;
                cols.clear();
                for (int64_t c = 0; c < span; c++)
                    if (mark[c]) cols.push_back((int32_t)(clo + c));
            } else {
                cols.assign(P.m_col.begin() + n0, P.m_col.begin() + n1);
                std::sort(cols.begin(), cols.end());
                cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
            }
            std::vector<int32_t> w;
            int64_t bytes = 0;
            int32_t a = cols[0];
            for (size_t k = 1; k <= cols.size(); k++) {
                if (k == cols.size() || cols[k] - cols[k - 1] > kWinGap) {
                    w.push_back(a);
                    w.push_back(cols[k - 1] + 1);
                    bytes += span16(cols[k - 1] + 1 - a, 4);
                    if (k < cols.size()) a = cols[k];
                }
            }
            const int64_t nw = (int64_t)w.size() / 2;
            if (nw > kMaxWin || bytes > work16(n1 - n0, 4)) return;
            int64_t off = 0;
            for (int64_t q = 0; q < nw; q++) {
                for (int32_t v : {w[2 * q], w[2 * q + 1], (int32_t)off, k}) P.win.push_back(v);
                off += span16(w[2 * q + 1] - w[2 * q], 4);
            }
            P.rwin[4 * rec + 1] = here + (int32_t)nw;
            P.rwin[4 * rec + 2] = (int32_t)bytes;
            // each entry's float index into the level's x area: its window is
            // the first whose end lies past its column (binary search)
            wend.resize(nw);
            wbase.resize(nw);
            for (int64_t q = 0, base = 0; q < nw; q++) {
                wend[q] = w[2 * q + 1];
                wbase[q] = base + (w[2 * q] & 3) - w[2 * q];
                base += span16(w[2 * q + 1] - w[2 * q], 4) / 4;
            }
            for (int32_t e = n0; e < n1; e++) {
                const int32_t c = P.m_col[e];
                const int64_t q = std::upper_bound(wend.begin(), wend.end(), c) - wend.begin();
                P.lcol[e] = (int32_t)(wbase[q] + c);
            }
        };
        // footprints of the levels [0, below) truncated at `below` (the
        // deepest level also stages one ev per child infoset)
        auto truncated = [&](const std::vector<std::pair<int32_t, int32_t>> &lv, int32_t below) {
            for (int32_t d = below - 1; d >= 0; d--)
                for (int32_t j = lv[d].first; j < lv[d].second; j++) {
                    int64_t u = own[j];
                    if (d + 1 < below) {
                        for (int32_t q = P.inf_seq[j]; q < P.inf_seq[j + 1]; q++)
                            for (int32_t c = P.seq_child[q]; c < P.seq_child[q + 1]; c++) u += f[c];
                    } else {
                        u += 4 * (int64_t)(P.seq_child[P.inf_seq[j + 1]] - P.seq_child[P.inf_seq[j]]);
                    }
                    f[j] = u;
                }
        };
        // unit size: enough units for ~2 per resident CTA over the whole batch,
        // within the buffer.  (The arithmetic of a sequence does not depend on
        // how the game is cut: every sum runs in the same fixed order, so a game
        // gives the same results alone and inside a batch.)
        int64_t batch_raw = 0;
        for (int64_t g = 0; g < G; g++) batch_raw += raw_up[g];
        int64_t target = batch_raw / std::max<int64_t>(1, 2 * opt.slots);
        target = std::max(opt.min_item_bytes, std::min(target, opt.item_bytes));
        for (int64_t g = 0; g < G; g++) {
            const auto &lv = glv[g];
            const int32_t nl = (int32_t)lv.size();   // levels 0..nl-1; level 0 = the root pseudo-infoset
            // tiers, bottom up: each tier starts at the shallowest level whose
            // subtrees, truncated at the tier below, fit the target
            std::vector<int32_t> tops;
            std::vector<std::vector<int64_t>> top_f;   // truncated footprints of each tier's top level
            for (int32_t below = nl; below > 0;) {
                truncated(lv, below);
                const int64_t tier_target =
                    below == nl ? target : std::max<int64_t>(1024, target / std::max<int64_t>(1, opt.internal_div));
                int32_t c = -1;
                for (int32_t d = 0; d < below && c < 0; d++) {
                    int64_t mx = 0;
                    for (int32_t j = lv[d].first; j < lv[d].second; j++) mx = std::max(mx, f[j]);
                    if (mx + slack_per_level * (below - d) <= tier_target) c = d;
                }
                if (opt.flat && c > 0) c = below - 1;   // one level per tier until the rest fits one unit
                if (c < 0) c = below - 1;   // a single level per tier; wider units run unstaged
                tops.push_back(c);
                top_f.emplace_back(f.begin() + lv[c].first, f.begin() + lv[c].second);
                below = c;
            }
            std::reverse(tops.begin(), tops.end());
            std::reverse(top_f.begin(), top_f.end());
            const int32_t m = (int32_t)tops.size();
            P.game_tiers[g] = m;
            // units, top down: each tier packs, per parent unit, the parent's
            // child infosets at the tier's top level into consecutive groups
            struct Span {
                int32_t parent, a, b;
            };
            std::vector<Span> spans{{-1, lv[0].first, lv[0].second}}, next;
            for (int32_t i = 0; i < m; i++) {
                const int32_t top = tops[i], bot = (i + 1 < m) ? tops[i + 1] : nl;
                const int64_t tier_target =
                    bot == nl ? target : std::max<int64_t>(1024, target / std::max<int64_t>(1, opt.internal_div));
                const int64_t cap = std::max<int64_t>(tier_target - slack_per_level * (bot - top), 1);
                const std::vector<int64_t> &ft = top_f[i];
                next.clear();
                auto emit = [&](int32_t par, int32_t a, int32_t b) {
                    Unit u{(int32_t)g, top, 0, (int32_t)P.ranges.size(), 0, par, 0, i};
                    int32_t lo = a, hi = b;
                    int64_t fu = 0, fd = 0;
                    for (int32_t d = top; d < bot && lo < hi; d++) {
                        push_level(lo, hi);
                        const int32_t slo = P.inf_seq[lo], shi = P.inf_seq[hi];
                        fu += up_level_bytes(shi - slo, hi - lo, P.m_ptr[shi] - P.m_ptr[slo]);
                        fd += down_level_bytes(shi - slo, hi - lo);
                        u.nlvl++;
                        lo = P.seq_child[slo];
                        hi = P.seq_child[shi];
                    }
                    const int32_t id = (int32_t)P.units.size();
                    if (lo < hi && top + u.nlvl == bot) {
                        // the child units' top levels: staged ev of [lo, hi)
                        u.flags |= kInternal;
                        next.push_back({id, lo, hi});
                        for (int32_t v : {lo, hi, 0, 0, 0, 0}) P.ranges.push_back(v);
                        for (int k = 0; k < 4; k++) P.rwin.push_back(0);
                        fu += span16(hi - lo, 4);
                    }
                    if (u.nlvl < kMaxStagedLevels && fu <= opt.item_bytes && fd <= opt.item_bytes) {
                        u.flags |= kStaged;
                        // x windows never take more room than the gathers
                        // the footprint above assumed
                        for (int32_t k = 0; k < u.nlvl; k++) {
                            const int32_t *r = &P.ranges[u.rng + kLvl * k];
                            windows(u.rng / kLvl + k, k, r[4], r[5]);
                        }
                    }
                    if (par >= 0) {
                        P.units[par].nchild++;
                        if (P.units[par].parent < 0) u.flags |= kChildOfRoot;
                    } else {
                        P.game_root[g] = id;
                    }
                    P.units.push_back(u);
                };
                for (const Span &sp : spans) {
                    int32_t a = sp.a;
                    int64_t acc = 0;
                    for (int32_t j = sp.a; j < sp.b; j++) {
                        const int64_t fj = ft[j - lv[top].first];
                        if (acc > 0 && acc + fj > cap) {
                            emit(sp.parent, a, j);
                            a = j;
                            acc = 0;
                        }
                        acc += fj;
                    }
                    emit(sp.parent, a, sp.b);
                }
                spans.swap(next);
            }
        }
        // top-down units: consecutive siblings (same parent, so adjacent
        // ranges at every level) merged while their top-down footprint fits.
        // A top-down unit also carries its ancestor chain: the infosets above
        // its top level, one contiguous range per level up to the game's root
        // (the parents of a contiguous range of infosets are one contiguous
        // range of sequences, since infosets are sorted by parent), staged
        // first as levels that are computed but not written back.  So the
        // unit rebuilds the next x of its top level's parents itself and
        // depends on no other top-down unit.
        {
            std::vector<int32_t> seq_inf(P.S);
            for (int64_t j = 0; j < J; j++)
                for (int32_t q = P.inf_seq[j]; q < P.inf_seq[j + 1]; q++) seq_inf[q] = (int32_t)j;
            std::vector<std::pair<int32_t, int32_t>> chain;
            auto ancestors = [&](int32_t lo, int32_t hi) {
                chain.clear();
                while (lo < hi && P.inf_par[lo] >= 0) {
                    const int32_t ps0 = P.inf_par[lo], ps1 = P.inf_par[hi - 1] + 1;
                    lo = seq_inf[ps0];
                    hi = seq_inf[ps1 - 1] + 1;
                    chain.push_back({lo, hi});
                }
                std::reverse(chain.begin(), chain.end());
                int64_t bytes = 0;
                for (auto &c : chain) bytes += down_level_bytes(P.inf_seq[c.second] - P.inf_seq[c.first], c.second - c.first);
                return bytes;
            };
            const int64_t nu0 = (int64_t)P.units.size();
            std::vector<int32_t> down_of(nu0, -1);
            P.dunits.clear();
            P.danc_off.clear();
            P.xanc_size = 0;
            auto build = [&](int64_t a, int64_t b) {   // up units [a, b), all siblings
                const Unit &f = P.units[a];
                Unit d{f.game, f.lvl0, 0, (int32_t)P.ranges.size(), 0, -1, 0, f.depth};
                int32_t lo = P.ranges[f.rng], hi = P.ranges[P.units[b - 1].rng + 1];
                int32_t nl = 0;
                for (int64_t k = a; k < b; k++) nl = std::max(nl, P.units[k].nlvl);
                int64_t fd = ancestors(lo, hi);
                int64_t anc_seqs = 0;
                for (auto &c : chain) {
                    push_level(c.first, c.second);
                    anc_seqs += P.inf_seq[c.second] - P.inf_seq[c.first];
                }
                const int32_t n_anc = (int32_t)chain.size();
                d.nlvl = n_anc;
                for (int32_t k = 0; k < nl && lo < hi; k++) {
                    push_level(lo, hi);
                    const int32_t slo = P.inf_seq[lo], shi = P.inf_seq[hi];
                    fd += down_level_bytes(shi - slo, hi - lo);
                    d.nlvl++;
                    lo = P.seq_child[slo];
                    hi = P.seq_child[shi];
                }
                if (d.nlvl < kMaxStagedLevels && fd <= opt.item_bytes) d.flags |= kStaged;
                d.flags |= n_anc << kAncShift;
                // a unit worked from global memory (unstaged, or any unit in
                // FP64) keeps its ancestors' x in a scratch area of its own
                P.danc_off.push_back((int32_t)P.xanc_size);
                P.xanc_size += anc_seqs;
                const int32_t up_par = f.parent;
                if (up_par >= 0) {
                    d.parent = down_of[up_par];
                    P.dunits[d.parent].nchild++;
                    if (P.units[up_par].parent < 0) d.flags |= kChildOfRoot;
                }
                const int32_t id = (int32_t)P.dunits.size();
                for (int64_t k = a; k < b; k++) down_of[k] = id;
                P.dunits.push_back(d);
            };
            auto fdown = [&](const Unit &u) {
                int64_t fd = 0;
                for (int32_t k = 0; k < u.nlvl; k++) {
                    const int32_t *r = &P.ranges[u.rng + kLvl * k];
                    fd += down_level_bytes(r[3] - r[2], r[1] - r[0]);
                }
                return fd;
            };
            // the ancestor chain of merged siblings [a, k]
            auto chain_bytes = [&](int64_t a, int64_t k) -> int64_t {
                return ancestors(P.ranges[P.units[a].rng], P.ranges[P.units[k].rng + 1]);
            };
            // runs of siblings merged while their footprint stays within cap;
            // emit(a, b) takes each run
            std::vector<int64_t> fdu(nu0);
            for (int64_t k = 0; k < nu0; k++) fdu[k] = fdown(P.units[k]);
            auto merge = [&](int64_t cap, auto &&emit_run) {
                int64_t a = 0, acc = 0;
                for (int64_t k = 0; k < nu0; k++) {
                    const Unit &u = P.units[k];
                    const bool same = k > a && u.game == P.units[a].game && u.parent == P.units[a].parent &&
                                      u.parent >= 0 && u.lvl0 == P.units[a].lvl0;
                    if (!same || acc + fdu[k] + chain_bytes(a, k) > cap) {
                        if (k > a) emit_run(a, k);
                        a = k;
                        acc = 0;
                    }
                    acc += fdu[k];
                }
                if (nu0 > a) emit_run(a, nu0);
            };
            // the smallest cap (within the buffer) that still gives no more
            // units than resident CTAs: top-down units are independent, so
            // the pass is then one round of CTAs with the most parallelism.
            // The count is estimated without the ancestor chains (cheap: one
            // pass over the units per probe), aiming a little under the CTAs.
            auto estimate = [&](int64_t cap) {
                int64_t n = 0, acc = 0, a = 0;
                for (int64_t k = 0; k < nu0; k++) {
                    const Unit &u = P.units[k];
                    const bool same = k > a && u.game == P.units[a].game && u.parent == P.units[a].parent &&
                                      u.parent >= 0 && u.lvl0 == P.units[a].lvl0;
                    if (!same || acc + fdu[k] > cap) {
                        n++;
                        a = k;
                        acc = 0;
                    }
                    acc += fdu[k];
                }
                return n;
            };
            const int64_t want = std::max<int64_t>(1, opt.slots * 7 / 8);
            int64_t lo_cap = opt.min_item_bytes, hi_cap = opt.item_bytes;
            if (estimate(hi_cap) <= want) {
                while (hi_cap - lo_cap > 1024) {
                    const int64_t mid = (lo_cap + hi_cap) / 2;
                    (estimate(mid) <= want ? hi_cap : lo_cap) = mid;
                }
            }
            merge(hi_cap, build);
        }
        // queues: leaves largest first for the bottom-up passes (a dynamic
        // queue then finishes with small units); every unit by tree depth for
        // the top-down pass, so a unit's parent always comes first
        const int64_t nu = (int64_t)P.units.size();
        std::vector<int64_t> usz(nu);
        for (int64_t k = 0; k < nu; k++) {
            const Unit &u = P.units[k];
            int64_t s = 0;
            for (int32_t d = 0; d < u.nlvl; d++)
                s += P.ranges[u.rng + kLvl * d + 3] - P.ranges[u.rng + kLvl * d + 2] +
                     P.ranges[u.rng + kLvl * d + 5] - P.ranges[u.rng + kLvl * d + 4];
            usz[k] = s;
        }
        // bottom-up queue: every leaf, largest first, then the internal units
        // deepest first, so a unit is always taken after all its children
        P.up_queue.clear();
        const int64_t nd = (int64_t)P.dunits.size();
        std::vector<int64_t> dsz(nd);
        for (int64_t k = 0; k < nd; k++) {
            const Unit &u = P.dunits[k];
            int64_t s = 0;
            for (int32_t d = 0; d < u.nlvl; d++)
                s += P.ranges[u.rng + kLvl * d + 3] - P.ranges[u.rng + kLvl * d + 2];
            dsz[k] = s;
        }
        P.down_queue.resize(nd);
        std::iota(P.down_queue.begin(), P.down_queue.end(), 0);
        std::vector<int32_t> internal;
        for (int64_t k = 0; k < nu; k++)
            (P.units[k].nchild == 0 ? P.up_queue : internal).push_back((int32_t)k);
        if (opt.leaf_order == 0)
            std::stable_sort(P.up_queue.begin(), P.up_queue.end(),
                             [&](int32_t a, int32_t b) { return usz[a] > usz[b]; });
        std::stable_sort(internal.begin(), internal.end(), [&](int32_t a, int32_t b) {
            if (P.units[a].depth != P.units[b].depth) return P.units[a].depth > P.units[b].depth;
            return usz[a] > usz[b];
        });
        P.up_queue.insert(P.up_queue.end(), internal.begin(), internal.end());
        std::stable_sort(P.down_queue.begin(), P.down_queue.end(), [&](int32_t a, int32_t b) {
            if (P.dunits[a].depth != P.dunits[b].depth) return P.dunits[a].depth < P.dunits[b].depth;
            return dsz[a] > dsz[b];
        });
    }
    L.game_nnz.assign(G, 0);
    for (int64_t r = 0; r < L.pl[0].S; r++)
        L.game_nnz[L.pl[0].seq_game[r]] += L.pl[0].m_ptr[r + 1] - L.pl[0].m_ptr[r];
    return ST_OK;
}

}  // namespace cfrb
