"""Independent formulations that pin the oracle (test-side only).

None of this code is shared with the oracle or with the CUDA path; each
function rebuilds what it needs from the raw tree arrays:

* ``SeqForm``       sequence-form objects (E, e, F, f, payoff matrix M) from
                    their definitions (von Stengel / Koller et al., Sec. 2.1).
* ``lp_value``      game value and equilibrium from the sequence-form LP.
* ``brute_force``   value of the reduced normal form (pure sequence-form
                    strategies enumerated) by the matrix-game LP.
* ``ClassicalCFR``  tree-walk CFR (Zinkevich et al.), which the paper states
                    produces the same iterates as sequence-form CFR (Sec. 2.1).
* ``Alg2``          the paper's Alg. 2 written with explicit logic matrices
                    A, B, C and level graphs L^(d) in scipy.sparse (Sec. 3.1-3.3).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog

CHANCE, P1, P2, TERMINAL = 0, 1, 2, 3


class SeqForm:
    """Sequence form of a tree in the caller's (infoset, action) order.

    Sequence numbering: 0 = empty, 1 + off[j] + a for (j, a)."""

    def __init__(self, tree):
        self.tree = tree
        n = tree.n_nodes
        kids = [[] for _ in range(n)]
        for i in range(1, n):
            kids[tree.parent[i]].append(i)
        for q in range(n):
            kids[q].sort(key=lambda c: tree.action[c])
        self.kids = kids
        self.nact = {}
        self.off = {}
        self.S = {}
        for p in (P1, P2):
            J = int(tree.infoset[tree.kind == p].max()) + 1 if (tree.kind == p).any() else 0
            na = np.zeros(J, dtype=int)
            for i in np.nonzero(tree.kind == p)[0]:
                na[tree.infoset[i]] = len(kids[i])
            self.nact[p] = na
            self.off[p] = np.concatenate([[0], np.cumsum(na)[:-1]]).astype(int) if J else np.zeros(0, int)
            self.S[p] = int(na.sum())
        # own sequence per node and chance reach
        seq = {P1: np.zeros(n, dtype=int), P2: np.zeros(n, dtype=int)}
        reach = np.ones(n)
        stack = [0]
        order = []
        while stack:
            q = stack.pop()
            order.append(q)
            for c in kids[q]:
                for p in (P1, P2):
                    if tree.kind[q] == p:
                        seq[p][c] = 1 + self.off[p][tree.infoset[q]] + tree.action[c]
                    else:
                        seq[p][c] = seq[p][q]
                reach[c] = reach[q] * (tree.chance_prob[c] if tree.kind[q] == CHANCE else 1.0)
                stack.append(c)
        self.seq = seq
        self.reach = reach
        self.par = {}
        for p in (P1, P2):
            J = len(self.nact[p])
            par = np.full(J, -1)
            for i in np.nonzero(tree.kind == p)[0]:
                par[tree.infoset[i]] = seq[p][i]
            self.par[p] = par
        S1, S2 = self.S[P1], self.S[P2]
        M = np.zeros((S1 + 1, S2 + 1))
        for z in np.nonzero(tree.kind == TERMINAL)[0]:
            M[seq[P1][z], seq[P2][z]] += reach[z] * tree.payoff[z]
        self.M = M

    def constraints(self, p):
        """E x = e: row 0 is x[empty] = 1, row 1 + j is sum_a x[(j,a)] - x[p_j] = 0."""
        J = len(self.nact[p])
        E = np.zeros((J + 1, self.S[p] + 1))
        E[0, 0] = 1.0
        for j in range(J):
            E[1 + j, self.par[p][j]] -= 1.0
            for a in range(self.nact[p][j]):
                E[1 + j, 1 + self.off[p][j] + a] += 1.0
        e = np.zeros(J + 1)
        e[0] = 1.0
        return E, e

    def seq_of(self, p, b):
        """sequence form of a behavioural strategy b (length S_p, caller order)"""
        J = len(self.nact[p])
        x = np.zeros(self.S[p] + 1)
        x[0] = 1.0
        done = np.zeros(J, bool)
        # parents first: repeat passes until all set (small trees only)
        while not done.all():
            for j in range(J):
                if done[j]:
                    continue
                ps = self.par[p][j]
                if ps == 0 or done[self._inf_of(p, ps)]:
                    for a in range(self.nact[p][j]):
                        s = self.off[p][j] + a
                        x[1 + s] = x[ps] * b[s]
                    done[j] = True
        return x

    def _inf_of(self, p, s):
        k = s - 1
        return int(np.searchsorted(self.off[p], k, side="right") - 1)


def lp_value(sf: SeqForm):
    """max_{x,z} f^T z  s.t.  E x = e, x >= 0, F^T z - M^T x <= 0 (z free).

    Returns (value, x*, y*) with y* from the symmetric LP of player 2."""
    E, e = sf.constraints(P1)
    F, f = sf.constraints(P2)
    M = sf.M
    n1, m2 = E.shape[1], F.shape[0]
    # variables [x (n1), z (m2)]; minimise -f^T z
    c = np.concatenate([np.zeros(n1), -f])
    A_ub = np.hstack([-M.T, F.T])
    b_ub = np.zeros(M.shape[1])
    A_eq = np.hstack([E, np.zeros((E.shape[0], m2))])
    bounds = [(0, None)] * n1 + [(None, None)] * m2
    r1 = linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=e, bounds=bounds, method="highs")
    assert r1.status == 0, r1.message
    v = -r1.fun
    x = r1.x[:n1]
    # player 2: min_{y,w} e^T w  s.t.  F y = f, y >= 0, E^T w - M y >= 0
    n2, m1 = F.shape[1], E.shape[0]
    c2 = np.concatenate([np.zeros(n2), e])
    A_ub2 = np.hstack([M, -E.T])
    b_ub2 = np.zeros(M.shape[0])
    A_eq2 = np.hstack([F, np.zeros((F.shape[0], m1))])
    bounds2 = [(0, None)] * n2 + [(None, None)] * m1
    r2 = linprog(c2, A_ub=A_ub2, b_ub=b_ub2, A_eq=A_eq2, b_eq=f, bounds=bounds2, method="highs")
    assert r2.status == 0, r2.message
    y = r2.x[:n2]
    return v, x, y


def _pure_strategies(sf: SeqForm, p):
    """All reduced pure strategies as 0/1 sequence-form vectors."""
    J = len(sf.nact[p])
    children = {}
    for j in range(J):
        children.setdefault(int(sf.par[p][j]), []).append(j)

    def expand(active_seqs):
        # infosets reachable under the chosen sequences
        infs = [j for s in active_seqs for j in children.get(s, [])]
        return infs

    out = []

    def rec(frontier, chosen):
        if not frontier:
            x = np.zeros(sf.S[p] + 1)
            x[0] = 1.0
            for s in chosen:
                x[s] = 1.0
            out.append(x)
            return
        j = frontier[0]
        for a in range(sf.nact[p][j]):
            s = 1 + sf.off[p][j] + a
            rec(frontier[1:] + children.get(s, []), chosen + [s])

    rec(list(children.get(0, [])), [])
    return out


def brute_force(sf: SeqForm):
    """Game value of the reduced normal form, by the matrix-game LP."""
    X = _pure_strategies(sf, P1)
    Y = _pure_strategies(sf, P2)
    N = np.array([[x @ sf.M @ y for y in Y] for x in X])
    m, n = N.shape
    # max v s.t. N^T p >= v, sum p = 1, p >= 0 ; variables [p, v]
    c = np.concatenate([np.zeros(m), [-1.0]])
    A_ub = np.hstack([-N.T, np.ones((n, 1))])
    b_ub = np.zeros(n)
    A_eq = np.concatenate([np.ones(m), [0.0]])[None, :]
    r = linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=[1.0],
                bounds=[(0, None)] * m + [(None, None)], method="highs")
    assert r.status == 0
    return -r.fun, len(X), len(Y)


class ClassicalCFR:
    """Tree-walk CFR over histories (regret/average tables per infoset).

    variant: 'cfr', 'cfr+', 'dcfr', 'pcfr+', 'pcfr'; the predictive step uses the
    instantaneous counterfactual regret of the last traversal (the prediction
    m = last utility valued under the last strategy)."""

    def __init__(self, tree):
        self.t = tree
        n = tree.n_nodes
        self.kids = [[] for _ in range(n)]
        for i in range(1, n):
            self.kids[tree.parent[i]].append(i)
        for q in range(n):
            self.kids[q].sort(key=lambda c: tree.action[c])
        self.R = {}
        self.avg = {}
        self.sigma = {}
        self.iter = 0
        for i in range(n):
            k = tree.kind[i]
            if k in (P1, P2):
                key = (int(k), int(tree.infoset[i]))
                na = len(self.kids[i])
                self.R[key] = np.zeros(na)
                self.avg[key] = np.zeros(na)
                self.sigma[key] = np.full(na, 1.0 / na)

    @staticmethod
    def rm(r):
        rp = np.maximum(r, 0.0)
        s = rp.sum()
        return rp / s if s > 0 else np.full(len(r), 1.0 / len(r))

    def _walk(self, h, pi, player, inst, w):
        """value of history h to `player`; pi = (chance, p1, p2) reach."""
        T = self.t
        k = T.kind[h]
        if k == TERMINAL:
            return T.payoff[h] if player == P1 else -T.payoff[h]
        if k == CHANCE:
            v = 0.0
            for c in self.kids[h]:
                v += T.chance_prob[c] * self._walk(c, (pi[0] * T.chance_prob[c], pi[1], pi[2]),
                                                   player, inst, w)
            return v
        key = (int(k), int(T.infoset[h]))
        s = self.sigma[key]
        vals = np.zeros(len(s))
        for a, c in enumerate(self.kids[h]):
            npi = list(pi)
            npi[k] *= s[a]
            vals[a] = self._walk(c, tuple(npi), player, inst, w)
        v = float(s @ vals)
        if k == player:
            opp = pi[0] * pi[P2 if player == P1 else P1]
            inst[key] = inst.get(key, 0.0) + opp * (vals - v)
            self.avg[key] += w * pi[player] * s
        return v

    def _update(self, player, variant, t, alpha, beta, gamma):
        inst = {}
        self._walk(0, (1.0, 1.0, 1.0), player, inst, t ** gamma)
        for key, d in inst.items():
            r = self.R[key] + d
            if variant in ("cfr+", "pcfr+"):
                r = np.maximum(r, 0.0)
            elif variant == "dcfr":
                fp = t ** alpha / (t ** alpha + 1)
                fn = t ** beta / (t ** beta + 1)
                r = np.where(r > 0, r * fp, np.where(r < 0, r * fn, r))
            self.R[key] = r
        for key, d in inst.items():
            if variant in ("pcfr+", "pcfr"):
                self.sigma[key] = self.rm(self.R[key] + d)
            else:
                self.sigma[key] = self.rm(self.R[key])

    def iterate(self, n, variant="cfr", alternating=False, alpha=1.5, beta=0.0, gamma=0.0):
        for _ in range(n):
            self.iter += 1
            t = float(self.iter)
            if alternating:
                self._update(P1, variant, t, alpha, beta, gamma)
                self._update(P2, variant, t, alpha, beta, gamma)
            else:
                # both traversals see the same profile: compute both increments first
                saved = {k: v.copy() for k, v in self.sigma.items()}
                inst = {}
                w = t ** gamma
                for p in (P1, P2):
                    d = {}
                    self._walk(0, (1.0, 1.0, 1.0), p, d, w)
                    inst[p] = d
                for p in (P1, P2):
                    for key, d in inst[p].items():
                        r = self.R[key] + d
                        if variant in ("cfr+", "pcfr+"):
                            r = np.maximum(r, 0.0)
                        elif variant == "dcfr":
                            fp = t ** alpha / (t ** alpha + 1)
                            fn = t ** beta / (t ** beta + 1)
                            r = np.where(r > 0, r * fp, np.where(r < 0, r * fn, r))
                        self.R[key] = r
                for p in (P1, P2):
                    for key, d in inst[p].items():
                        self.sigma[key] = self.rm(self.R[key] + d if variant in ("pcfr+", "pcfr") else self.R[key])
                del saved

    def regrets(self, p, sf: SeqForm):
        out = np.zeros(sf.S[p])
        for (q, j), r in self.R.items():
            if q == p:
                out[sf.off[p][j]: sf.off[p][j] + len(r)] = r
        return out

    def average(self, p, sf: SeqForm):
        out = np.zeros(sf.S[p])
        for (q, j), a in self.avg.items():
            if q == p:
                s = a.sum()
                out[sf.off[p][j]: sf.off[p][j] + len(a)] = a / s if s > 0 else 1.0 / len(a)
        return out


class Alg2:
    """Alg. 2 with explicit logic matrices and level graphs for one player.

    TFSDP nodes: the root observation point (rho(empty)), one decision point
    per infoset and one observation point rho(j, a) per sequence; decision
    points hang below the observation point of their parent sequence."""

    def __init__(self, sf: SeqForm, p):
        na, off, par = sf.nact[p], sf.off[p], sf.par[p]
        J, S = len(na), sf.S[p]
        # node ids: 0 = root obs, 1..J decision points, J+1..J+S observation points
        self.J, self.S = J, S
        P = 1 + J + S
        depth = np.zeros(P, dtype=int)
        # decision point j sits below obs node of par[j]
        obs_of_seq = lambda s: 0 if s == 0 else J + s        # sequence s (1-based) -> obs node
        # compute depths by walking parents
        dp_depth = np.full(J, -1)

        def ddepth(j):
            if dp_depth[j] >= 0:
                return dp_depth[j]
            ps = par[j]
            if ps == 0:
                d = 1
            else:
                jp = int(np.searchsorted(off, ps - 1, side="right") - 1)
                d = ddepth(jp) + 2
            dp_depth[j] = d
            return d

        for j in range(J):
            depth[1 + j] = ddepth(j)
            for a in range(na[j]):
                depth[J + 1 + off[j] + a] = depth[1 + j] + 1
        self.k = int(depth.max())
        # A: P x (S+1), A[p, s] = 1[p = rho(s)]
        rows = [0] + [J + 1 + s for s in range(S)]
        self.A = sp.csr_matrix((np.ones(S + 1), (rows, np.arange(S + 1))), shape=(P, S + 1))
        self.B = self.A[:, 1:]
        # C: J x S, C[j, (j', a)] = 1[j = j']
        crow = np.repeat(np.arange(J), na)
        self.C = sp.csr_matrix((np.ones(S), (crow, np.arange(S))), shape=(J, S))
        # level graphs: edges parent -> child at child depth d
        self.edges = []   # (parent node, child node, seq index or -1 for signal edge)
        for j in range(J):
            self.edges.append((obs_of_seq(par[j]), 1 + j, -1))
            for a in range(na[j]):
                s = off[j] + a
                self.edges.append((1 + j, J + 1 + s, s))
        self.depth = depth
        self.P = P

    def L(self, d, b):
        rows, cols, vals = [], [], []
        for (u, v, s) in self.edges:
            if self.depth[v] == d:
                rows.append(u)
                cols.append(v)
                vals.append(1.0 if s < 0 else b[s])
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.P, self.P))

    def next_strategy(self, r):
        rp = np.maximum(r, 0.0)
        den = self.C.T @ (self.C @ rp)
        na = np.asarray(self.C.sum(axis=1)).ravel()
        uni = self.C.T @ (1.0 / na)
        b = np.where(den > 0, rp / np.where(den > 0, den, 1.0), uni)
        y = np.zeros(self.P)
        y[0] = 1.0
        for d in range(1, self.k + 1):
            y = y + self.L(d, b).T @ y
        x = self.A.T @ y
        return b, x

    def observe_utility(self, u, b, r):
        v = np.zeros(self.P)
        w = self.A @ u
        for d in range(self.k, 0, -1):
            Ld = self.L(d, b)
            v = v + Ld @ w + Ld @ v
        q = self.B.T @ (w + v)
        r_new = r + q - self.C.T @ (self.C @ (b * q))
        return r_new, q
