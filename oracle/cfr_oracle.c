/*
 * Plain FP64 CPU oracle for sequence-form CFR -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the checker the CUDA path is compared against.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it;
 * the product library never does.  It shares no code with the CUDA path: it has
 * its own tree compiler, its own sequence numbering (the caller's
 * (infoset, action) order) and its own loops.
 *
 * What it computes, and where each step comes from ("Parallelizing
 * Counterfactual Regret Minimization", Kim & Sandholm):
 *
 *   - sequence form (Sec. 2.1): sigma = (j, a), empty sequence 0, parent
 *     sequence p_j of decision point j; x[0] = 1, x[(j,a)] = x[p_j] b_j[a].
 *   - NextStrategy (Alg. 1): regret matching b_j = (r_j)^+ / ||(r_j)^+||_1,
 *     uniform when the norm is 0 (the paper leaves that case "arbitrary"),
 *     then the top-down conversion to sequence form.
 *   - utilities (Sec. 2.1, two-player case): u1[s1] = sum_z pi_c(z) u1(z) y[s2(z)],
 *     u2[s2] = -sum_z pi_c(z) u1(z) x[s1(z)], one pass over the terminals.
 *   - ObserveUtility (Alg. 1): bottom-up counterfactual values
 *     V[(j,a)] = u[(j,a)] + sum_{j': p_j' = (j,a)} ev_j',  ev_j = sum_a b_j[a] V[(j,a)]
 *     (observation points sum their children with weight 1), then
 *     r_j += V[(j,.)] - ev_j.
 *   - CFR+ (Alg. 3): r := r^+ after ObserveUtility.
 *   - DCFR (Alg. 4): r *= t^a/(t^a+1) where r > 0, t^b/(t^b+1) where r < 0.
 *   - PCFR+ (Alg. 5): NextStrategy*(m) with m = the last utility: back up r,
 *     keep the previous behavioural strategy, ObserveUtility(m), regret
 *     matching, restore r.  Regrets are floored as in CFR+.
 *   - PCFR (Sec. 3.5.4, the predictive counterpart of CFR): the same
 *     NextStrategy*(m), with regrets never floored (no post-op).
 *   - alternating updates (Sec. 3.5.1): player 2's half-step sees player 1's
 *     strategy recomputed after player 1's update.
 *   - average strategy: xbar += t^gamma x^t for the strategy played at t.
 *   - exploitability (Sec. 4 uses it without a definition): best responses
 *     to the normalised averages, (BR1 + BR2) / 2.
 *
 * Build: gcc -O2 -shared -fPIC -o liboracle.so cfr_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OK 0
#define ERR_INVALID (-1)
#define ERR_OOM (-2)
#define ERR_STATE (-5)

enum { K_CHANCE = 0, K_P1 = 1, K_P2 = 2, K_TERM = 3 };
enum { V_CFR = 0, V_CFRPLUS = 1, V_DCFR = 2, V_PCFRPLUS = 3, V_PCFR = 4 };

typedef struct {
    int64_t J;          /* infosets */
    int64_t S;          /* non-empty sequences; arrays indexed 0..S, 0 = empty */
    int32_t *nact;      /* [J] actions of infoset j */
    int64_t *off;       /* [J] sequence index of (j, 0) */
    int64_t *par;       /* [J] parent sequence p_j */
    int64_t *topo;      /* [J] infosets, parents before children */
    int64_t *cptr;      /* [S+2] child infosets of sequence s: cinf[cptr[s]..cptr[s+1]) */
    int64_t *cinf;
    double *r, *b, *xbar; /* state: r[S+1], b[S+1], xbar[S+1] */
} player_t;

typedef struct {
    player_t pl[3];     /* index 1 and 2 */
    int64_t nterm;
    int64_t *ts1, *ts2; /* sequence of each player leading to terminal z */
    double *tw;         /* pi_c(z) * u1(z) */
    int64_t t;          /* completed iterations */
} oracle_game;

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

static void free_player(player_t *p) {
    free(p->nact); free(p->off); free(p->par); free(p->topo);
    free(p->cptr); free(p->cinf); free(p->r); free(p->b); free(p->xbar);
}

void oracle_free(oracle_game *g) {
    if (!g) return;
    free_player(&g->pl[1]);
    free_player(&g->pl[2]);
    free(g->ts1); free(g->ts2); free(g->tw);
    free(g);
}

/* ---------------------------------------------------------------------------
 * tree -> sequence form
 * ------------------------------------------------------------------------- */
int oracle_build(int64_t n, const int32_t *parent, const int8_t *kind, const int32_t *infoset,
                 const int32_t *action, const double *chance_prob, const double *payoff,
                 oracle_game **out) {
    *out = NULL;
    if (n < 1 || parent[0] != -1) return ERR_INVALID;
    oracle_game *g = (oracle_game *)xcalloc(1, sizeof(oracle_game));
    int rc = ERR_INVALID;
    int64_t *nch = (int64_t *)xcalloc(n, sizeof(int64_t));
    int64_t *seq[3] = {0, 0, 0};
    seq[1] = (int64_t *)xcalloc(n, sizeof(int64_t));
    seq[2] = (int64_t *)xcalloc(n, sizeof(int64_t));
    double *pc = (double *)xcalloc(n, sizeof(double));
    double *psum = (double *)xcalloc(n, sizeof(double));
    int64_t *lvl = NULL, *seq_inf = NULL;
    if (!g || !nch || !seq[1] || !seq[2] || !pc || !psum) { rc = ERR_OOM; goto fail; }

    /* structural checks and child counts */
    for (int64_t i = 0; i < n; i++) {
        if (kind[i] < 0 || kind[i] > 3) goto fail;
        if (i > 0) {
            if (parent[i] < 0 || parent[i] >= i) goto fail;
            if (kind[parent[i]] == K_TERM) goto fail;
            nch[parent[i]]++;
        }
        if ((kind[i] == K_P1 || kind[i] == K_P2) && infoset[i] < 0) goto fail;
        if (kind[i] == K_TERM && !isfinite(payoff[i])) goto fail;
    }
    for (int64_t i = 0; i < n; i++)
        if (kind[i] != K_TERM && nch[i] == 0) goto fail;
    /* action labels: each parent's children carry 0..nch-1 exactly once;
     * chance probabilities lie in [0,1] and sum to 1 */
    {
        int64_t *coff = (int64_t *)xcalloc(n + 1, sizeof(int64_t));
        unsigned char *seen = (unsigned char *)xcalloc(n, 1);
        if (!coff || !seen) { free(coff); free(seen); rc = ERR_OOM; goto fail; }
        for (int64_t i = 0; i < n; i++) coff[i + 1] = coff[i] + nch[i];
        int bad = 0;
        for (int64_t i = 1; i < n && !bad; i++) {
            int64_t q = parent[i];
            if (action[i] < 0 || action[i] >= nch[q]) { bad = 1; break; }
            if (seen[coff[q] + action[i]]) { bad = 1; break; }
            seen[coff[q] + action[i]] = 1;
            if (kind[q] == K_CHANCE) {
                if (!(chance_prob[i] >= 0.0 && chance_prob[i] <= 1.0)) { bad = 1; break; }
                psum[q] += chance_prob[i];
            }
        }
        free(coff); free(seen);
        if (bad) goto fail;
        for (int64_t i = 0; i < n; i++)
            if (kind[i] == K_CHANCE && fabs(psum[i] - 1.0) > 1e-9) goto fail;
    }

    /* infoset sizes and action counts */
    for (int p = 1; p <= 2; p++) {
        int64_t J = 0;
        for (int64_t i = 0; i < n; i++)
            if (kind[i] == p && infoset[i] + 1 > J) J = infoset[i] + 1;
        player_t *P = &g->pl[p];
        P->J = J;
        P->nact = (int32_t *)xcalloc(J, sizeof(int32_t));
        P->off = (int64_t *)xcalloc(J, sizeof(int64_t));
        P->par = (int64_t *)xcalloc(J, sizeof(int64_t));
        P->topo = (int64_t *)xcalloc(J, sizeof(int64_t));
        if (!P->nact || !P->off || !P->par || !P->topo) { rc = ERR_OOM; goto fail; }
        for (int64_t j = 0; j < J; j++) P->par[j] = -1;
        for (int64_t i = 0; i < n; i++) {
            if (kind[i] != p) continue;
            int64_t j = infoset[i];
            if (P->nact[j] == 0) P->nact[j] = (int32_t)nch[i];
            else if (P->nact[j] != nch[i]) goto fail;          /* action-count mismatch */
        }
        int64_t s = 1;
        for (int64_t j = 0; j < J; j++) {
            if (P->nact[j] == 0) goto fail;                     /* ids must be dense */
            P->off[j] = s;
            s += P->nact[j];
        }
        P->S = s - 1;
    }

    /* own sequence at every node and chance reach, top-down */
    pc[0] = 1.0;
    for (int64_t i = 1; i < n; i++) {
        int64_t q = parent[i];
        for (int p = 1; p <= 2; p++)
            seq[p][i] = (kind[q] == p) ? g->pl[p].off[infoset[q]] + action[i] : seq[p][q];
        pc[i] = pc[q] * ((kind[q] == K_CHANCE) ? chance_prob[i] : 1.0);
    }

    /* parent sequence of each infoset; perfect recall = all its nodes agree */
    for (int64_t i = 0; i < n; i++) {
        int p = kind[i];
        if (p != K_P1 && p != K_P2) continue;
        player_t *P = &g->pl[p];
        int64_t j = infoset[i];
        if (P->par[j] < 0) P->par[j] = seq[p][i];
        else if (P->par[j] != seq[p][i]) goto fail;
    }

    /* levels, topological order and child lists */
    for (int p = 1; p <= 2; p++) {
        player_t *P = &g->pl[p];
        int64_t J = P->J, S = P->S;
        seq_inf = (int64_t *)xcalloc(S + 1, sizeof(int64_t));
        lvl = (int64_t *)xcalloc(J, sizeof(int64_t));
        P->cptr = (int64_t *)xcalloc(S + 2, sizeof(int64_t));
        P->cinf = (int64_t *)xcalloc(J, sizeof(int64_t));
        P->r = (double *)xcalloc(S + 1, sizeof(double));
        P->b = (double *)xcalloc(S + 1, sizeof(double));
        P->xbar = (double *)xcalloc(S + 1, sizeof(double));
        if (!seq_inf || !lvl || !P->cptr || !P->cinf || !P->r || !P->b || !P->xbar) {
            rc = ERR_OOM; goto fail;
        }
        seq_inf[0] = -1;
        for (int64_t j = 0; j < J; j++)
            for (int a = 0; a < P->nact[j]; a++) seq_inf[P->off[j] + a] = j;
        /* level by repeated relaxation: a parent sequence's infoset always has
         * a strictly smaller level, and parents can be found by walking up */
        for (int64_t j = 0; j < J; j++) {
            int64_t d = 1, s = P->par[j];
            while (s != 0) {
                d++;
                s = P->par[seq_inf[s]];
                if (d > J + 1) goto fail;                       /* cycle */
            }
            lvl[j] = d;
        }
        /* counting sort by level, stable in infoset id */
        int64_t maxl = 0;
        for (int64_t j = 0; j < J; j++) if (lvl[j] > maxl) maxl = lvl[j];
        int64_t *cnt = (int64_t *)xcalloc(maxl + 2, sizeof(int64_t));
        if (!cnt) { rc = ERR_OOM; goto fail; }
        for (int64_t j = 0; j < J; j++) cnt[lvl[j] + 1]++;
        for (int64_t l = 1; l <= maxl + 1; l++) cnt[l] += cnt[l - 1];
        for (int64_t j = 0; j < J; j++) P->topo[cnt[lvl[j]]++] = j;
        free(cnt);
        /* children of each sequence (CSR over sequence index) */
        for (int64_t j = 0; j < J; j++) P->cptr[P->par[j] + 1]++;
        for (int64_t s = 1; s <= S + 1; s++) P->cptr[s] += P->cptr[s - 1];
        int64_t *fill = (int64_t *)xcalloc(S + 1, sizeof(int64_t));
        if (!fill) { rc = ERR_OOM; goto fail; }
        for (int64_t j = 0; j < J; j++) {
            int64_t s = P->par[j];
            P->cinf[P->cptr[s] + fill[s]++] = j;
        }
        free(fill);
        free(seq_inf); seq_inf = NULL;
        free(lvl); lvl = NULL;
        /* initial state: r = 0, b = uniform */
        for (int64_t j = 0; j < J; j++)
            for (int a = 0; a < P->nact[j]; a++) P->b[P->off[j] + a] = 1.0 / P->nact[j];
    }

    /* terminals */
    {
        int64_t nt = 0;
        for (int64_t i = 0; i < n; i++) nt += (kind[i] == K_TERM);
        g->nterm = nt;
        g->ts1 = (int64_t *)xcalloc(nt, sizeof(int64_t));
        g->ts2 = (int64_t *)xcalloc(nt, sizeof(int64_t));
        g->tw = (double *)xcalloc(nt, sizeof(double));
        if (!g->ts1 || !g->ts2 || !g->tw) { rc = ERR_OOM; goto fail; }
        int64_t z = 0;
        for (int64_t i = 0; i < n; i++) {
            if (kind[i] != K_TERM) continue;
            g->ts1[z] = seq[1][i];
            g->ts2[z] = seq[2][i];
            g->tw[z] = pc[i] * payoff[i];
            z++;
        }
    }
    g->t = 0;
    free(nch); free(seq[1]); free(seq[2]); free(pc); free(psum);
    *out = g;
    return OK;
fail:
    free(nch); free(seq[1]); free(seq[2]); free(pc); free(psum);
    free(lvl); free(seq_inf);
    oracle_free(g);
    return rc;
}

int oracle_sizes(const oracle_game *g, int64_t *out) {
    out[0] = g->pl[1].S; out[1] = g->pl[2].S;
    out[2] = g->pl[1].J; out[3] = g->pl[2].J;
    out[4] = g->nterm;   out[5] = g->t;
    return OK;
}

/* ---------------------------------------------------------------------------
 * the steps of one iteration
 * ------------------------------------------------------------------------- */

/* NextStrategy, first half (Alg. 1): regret matching per decision point */
static void regret_matching(const player_t *P, const double *r, double *b) {
    for (int64_t j = 0; j < P->J; j++) {
        int64_t o = P->off[j];
        int na = P->nact[j];
        double s = 0.0;
        for (int a = 0; a < na; a++) s += r[o + a] > 0.0 ? r[o + a] : 0.0;
        for (int a = 0; a < na; a++)
            b[o + a] = (s > 0.0) ? (r[o + a] > 0.0 ? r[o + a] : 0.0) / s : 1.0 / na;
    }
}

/* NextStrategy, second half (Alg. 1): behavioural -> sequence form, top-down */
static void sequence_form(const player_t *P, const double *b, double *x) {
    x[0] = 1.0;
    for (int64_t k = 0; k < P->J; k++) {
        int64_t j = P->topo[k];
        for (int a = 0; a < P->nact[j]; a++) x[P->off[j] + a] = x[P->par[j]] * b[P->off[j] + a];
    }
}

/* sparse payoff product over the terminal list */
static void utility(const oracle_game *g, int p, const double *xo, double *u) {
    memset(u, 0, (size_t)(g->pl[p].S + 1) * sizeof(double));
    for (int64_t z = 0; z < g->nterm; z++) {
        if (p == 1) u[g->ts1[z]] += g->tw[z] * xo[g->ts2[z]];
        else u[g->ts2[z]] -= g->tw[z] * xo[g->ts1[z]];
    }
}

/* ObserveUtility (Alg. 1): bottom-up values, then r += V - ev.  V[S+1], ev[J]. */
static void observe_utility(const player_t *P, const double *u, const double *b, double *r,
                            double *V, double *ev) {
    for (int64_t k = P->J - 1; k >= 0; k--) {
        int64_t j = P->topo[k];
        double e = 0.0;
        for (int a = 0; a < P->nact[j]; a++) {
            int64_t s = P->off[j] + a;
            double v = u[s];
            for (int64_t c = P->cptr[s]; c < P->cptr[s + 1]; c++) v += ev[P->cinf[c]];
            V[s] = v;
            e += b[s] * v;
        }
        ev[j] = e;
    }
    for (int64_t j = 0; j < P->J; j++)
        for (int a = 0; a < P->nact[j]; a++) r[P->off[j] + a] += V[P->off[j] + a] - ev[j];
}

static void post_op(const player_t *P, int variant, double t, double alpha, double beta, double *r) {
    if (variant == V_CFRPLUS || variant == V_PCFRPLUS) {
        for (int64_t s = 1; s <= P->S; s++) r[s] = r[s] > 0.0 ? r[s] : 0.0;
    } else if (variant == V_DCFR) {
        double ta = pow(t, alpha), tb = pow(t, beta);
        double fp = ta / (ta + 1.0), fn = tb / (tb + 1.0);
        for (int64_t s = 1; s <= P->S; s++) {
            if (r[s] > 0.0) r[s] *= fp;
            else if (r[s] < 0.0) r[s] *= fn;
        }
    }
}

typedef struct { double *x, *u, *V, *ev, *rho; } scratch_t;

/* one player's update at iteration t: average, ObserveUtility, variant, next strategy */
static void update_player(oracle_game *g, int p, const double *u, const double *xplayed,
                          int variant, double t, double alpha, double beta, double gamma,
                          scratch_t *sc) {
    player_t *P = &g->pl[p];
    double w = pow(t, gamma);
    for (int64_t s = 0; s <= P->S; s++) P->xbar[s] += w * xplayed[s];
    observe_utility(P, u, P->b, P->r, sc->V, sc->ev);
    post_op(P, variant, t, alpha, beta, P->r);
    if (variant == V_PCFRPLUS || variant == V_PCFR) {
        /* NextStrategy*(m = u): back up r, observe the prediction with the
         * previous behavioural strategy, regret-match, restore r */
        memcpy(sc->rho, P->r, (size_t)(P->S + 1) * sizeof(double));
        observe_utility(P, u, P->b, P->r, sc->V, sc->ev);
        regret_matching(P, P->r, P->b);
        memcpy(P->r, sc->rho, (size_t)(P->S + 1) * sizeof(double));
    } else {
        regret_matching(P, P->r, P->b);
    }
}

int oracle_iterate(oracle_game *g, int64_t n, int variant, double alpha, double beta,
                   double gamma, int alternating) {
    if (variant < 0 || variant > 4 || n < 0) return ERR_INVALID;
    int64_t Smax = g->pl[1].S > g->pl[2].S ? g->pl[1].S : g->pl[2].S;
    int64_t Jmax = g->pl[1].J > g->pl[2].J ? g->pl[1].J : g->pl[2].J;
    double *x = (double *)xcalloc(g->pl[1].S + 1, sizeof(double));
    double *y = (double *)xcalloc(g->pl[2].S + 1, sizeof(double));
    double *u1 = (double *)xcalloc(g->pl[1].S + 1, sizeof(double));
    double *u2 = (double *)xcalloc(g->pl[2].S + 1, sizeof(double));
    scratch_t sc;
    sc.V = (double *)xcalloc(Smax + 1, sizeof(double));
    sc.ev = (double *)xcalloc(Jmax, sizeof(double));
    sc.rho = (double *)xcalloc(Smax + 1, sizeof(double));
    int rc = OK;
    if (!x || !y || !u1 || !u2 || !sc.V || !sc.ev || !sc.rho) { rc = ERR_OOM; goto done; }
    for (int64_t it = 0; it < n; it++) {
        double t = (double)(g->t + 1);
        sequence_form(&g->pl[1], g->pl[1].b, x);
        sequence_form(&g->pl[2], g->pl[2].b, y);
        if (!alternating) {
            utility(g, 1, y, u1);
            utility(g, 2, x, u2);
            update_player(g, 1, u1, x, variant, t, alpha, beta, gamma, &sc);
            update_player(g, 2, u2, y, variant, t, alpha, beta, gamma, &sc);
        } else {
            utility(g, 1, y, u1);
            update_player(g, 1, u1, x, variant, t, alpha, beta, gamma, &sc);
            sequence_form(&g->pl[1], g->pl[1].b, x);      /* player 2 sees the new x */
            utility(g, 2, x, u2);
            update_player(g, 2, u2, y, variant, t, alpha, beta, gamma, &sc);
        }
        g->t += 1;
    }
done:
    free(x); free(y); free(u1); free(u2); free(sc.V); free(sc.ev); free(sc.rho);
    return rc;
}

/* ---------------------------------------------------------------------------
 * best response and exploitability
 * ------------------------------------------------------------------------- */

/* value of player p's best response to the other player's sequence-form
 * strategy xo: V[s] = u[s] + sum_{children j} max_a V[(j,a)], BR = V[empty] */
static double best_response(const oracle_game *g, int p, const double *xo, double *u, double *V,
                            double *best) {
    const player_t *P = &g->pl[p];
    utility(g, p, xo, u);
    for (int64_t k = P->J - 1; k >= 0; k--) {
        int64_t j = P->topo[k];
        double m = -INFINITY;
        for (int a = 0; a < P->nact[j]; a++) {
            int64_t s = P->off[j] + a;
            double v = u[s];
            for (int64_t c = P->cptr[s]; c < P->cptr[s + 1]; c++) v += best[P->cinf[c]];
            V[s] = v;
            if (v > m) m = v;
        }
        best[j] = m;
    }
    double root = u[0];
    for (int64_t c = P->cptr[0]; c < P->cptr[1]; c++) root += best[P->cinf[c]];
    return root;
}

/* exploitability of an explicit profile (sequence form, length S_i + 1, [0] = 1) */
int oracle_exploitability_of(const oracle_game *g, const double *x, const double *y,
                             double *expl, double *br1, double *br2) {
    int64_t Smax = g->pl[1].S > g->pl[2].S ? g->pl[1].S : g->pl[2].S;
    int64_t Jmax = g->pl[1].J > g->pl[2].J ? g->pl[1].J : g->pl[2].J;
    double *u = (double *)xcalloc(Smax + 1, sizeof(double));
    double *V = (double *)xcalloc(Smax + 1, sizeof(double));
    double *best = (double *)xcalloc(Jmax, sizeof(double));
    if (!u || !V || !best) { free(u); free(V); free(best); return ERR_OOM; }
    double b1 = best_response(g, 1, y, u, V, best);
    double b2 = best_response(g, 2, x, u, V, best);
    free(u); free(V); free(best);
    *br1 = b1; *br2 = b2;
    *expl = 0.5 * (b1 + b2);
    return OK;
}

/* exploitability of the average profile xbar / xbar[empty] (current profile if t = 0) */
int oracle_exploitability(const oracle_game *g, double *expl, double *br1, double *br2) {
    double *xs[3] = {0, 0, 0};
    for (int p = 1; p <= 2; p++) {
        const player_t *P = &g->pl[p];
        xs[p] = (double *)xcalloc(P->S + 1, sizeof(double));
        if (!xs[p]) { free(xs[1]); return ERR_OOM; }
        if (P->xbar[0] > 0.0) {
            for (int64_t s = 0; s <= P->S; s++) xs[p][s] = P->xbar[s] / P->xbar[0];
        } else {
            sequence_form(P, P->b, xs[p]);
        }
    }
    int rc = oracle_exploitability_of(g, xs[1], xs[2], expl, br1, br2);
    free(xs[1]); free(xs[2]);
    return rc;
}

/* ---------------------------------------------------------------------------
 * state and single steps, all in the caller's (infoset, action) order:
 * r[S], b[S] hold sequence k = off[j] - 1 + a; xbar[S + 1] has the empty
 * sequence at [0] and sequence k at [1 + k].
 * ------------------------------------------------------------------------- */
int oracle_get_state(const oracle_game *g, int p, double *r, double *b, double *xbar, int64_t *t) {
    if (p != 1 && p != 2) return ERR_INVALID;
    const player_t *P = &g->pl[p];
    for (int64_t s = 1; s <= P->S; s++) { r[s - 1] = P->r[s]; b[s - 1] = P->b[s]; }
    for (int64_t s = 0; s <= P->S; s++) xbar[s] = P->xbar[s];
    *t = g->t;
    return OK;
}

int oracle_set_state(oracle_game *g, int p, const double *r, const double *b, const double *xbar,
                     int64_t t) {
    if ((p != 1 && p != 2) || t < 0) return ERR_INVALID;
    player_t *P = &g->pl[p];
    P->r[0] = 0.0; P->b[0] = 1.0;
    for (int64_t s = 1; s <= P->S; s++) { P->r[s] = r[s - 1]; P->b[s] = b[s - 1]; }
    for (int64_t s = 0; s <= P->S; s++) P->xbar[s] = xbar[s];
    g->t = t;
    return OK;
}

/* behavioural average: xbar[(j,a)] / xbar[p_j], uniform where xbar[p_j] = 0 */
int oracle_average_strategy(const oracle_game *g, int p, double *out) {
    if (p != 1 && p != 2) return ERR_INVALID;
    const player_t *P = &g->pl[p];
    for (int64_t j = 0; j < P->J; j++) {
        double d = P->xbar[P->par[j]];
        for (int a = 0; a < P->nact[j]; a++)
            out[P->off[j] - 1 + a] = d > 0.0 ? P->xbar[P->off[j] + a] / d : 1.0 / P->nact[j];
    }
    return OK;
}

int oracle_regret_matching(const oracle_game *g, int p, const double *r, double *b) {
    const player_t *P = &g->pl[p];
    double *rr = (double *)xcalloc(P->S + 1, sizeof(double));
    double *bb = (double *)xcalloc(P->S + 1, sizeof(double));
    if (!rr || !bb) { free(rr); free(bb); return ERR_OOM; }
    memcpy(rr + 1, r, (size_t)P->S * sizeof(double));
    regret_matching(P, rr, bb);
    memcpy(b, bb + 1, (size_t)P->S * sizeof(double));
    free(rr); free(bb);
    return OK;
}

/* sequence form of a behavioural strategy b[S] -> x[S + 1] */
int oracle_sequence_form(const oracle_game *g, int p, const double *b, double *x) {
    const player_t *P = &g->pl[p];
    double *bb = (double *)xcalloc(P->S + 1, sizeof(double));
    if (!bb) return ERR_OOM;
    memcpy(bb + 1, b, (size_t)P->S * sizeof(double));
    sequence_form(P, bb, x);
    free(bb);
    return OK;
}

/* utility of player p against the other player's sequence form xo[S_o + 1] -> u[S_p + 1] */
int oracle_utility(const oracle_game *g, int p, const double *xo, double *u) {
    if (p != 1 && p != 2) return ERR_INVALID;
    utility(g, p, xo, u);
    return OK;
}

/* ObserveUtility with explicit b and r (r updated in place, both length S);
 * u has length S + 1; V (S + 1) and ev (J) receive the counterfactual values */
int oracle_observe_utility(const oracle_game *g, int p, const double *u, const double *b,
                           double *r, double *V, double *ev) {
    const player_t *P = &g->pl[p];
    double *bb = (double *)xcalloc(P->S + 1, sizeof(double));
    double *rr = (double *)xcalloc(P->S + 1, sizeof(double));
    if (!bb || !rr) { free(bb); free(rr); return ERR_OOM; }
    memcpy(bb + 1, b, (size_t)P->S * sizeof(double));
    memcpy(rr + 1, r, (size_t)P->S * sizeof(double));
    memset(V, 0, (size_t)(P->S + 1) * sizeof(double));
    observe_utility(P, u, bb, rr, V, ev);
    memcpy(r, rr + 1, (size_t)P->S * sizeof(double));
    free(bb); free(rr);
    return OK;
}

/* structure queries used by the tests: parent sequence (caller numbering,
 * -1 = empty) and action count of every infoset */
int oracle_infosets(const oracle_game *g, int p, int64_t *parent_seq, int32_t *nact) {
    const player_t *P = &g->pl[p];
    for (int64_t j = 0; j < P->J; j++) {
        parent_seq[j] = P->par[j] - 1;
        nact[j] = P->nact[j];
    }
    return OK;
}
