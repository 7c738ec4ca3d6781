// n-player sequence-form CFR (include/cfr_nplayer.h): the utility step is the
// contraction of each player's payoff tensor with the other players'
// sequence-form strategies ("tensor operations in multiplayer settings",
// Sec. 2.1); every other step is the two-player path's per-infoset arithmetic
// (kernels.cuh: up_infoset_cfr's, with its loads issued together; up_infoset_br;
// the float-float sums).
//
// Layout per player (host compile below):
// * the player's decision points numbered level by level (a level's children
//   are the next level), within a level by parent sequence, then by the
//   caller's infoset id; sequences numbered by decision point, actions in
//   order; sequence 0 is the empty one.  So each decision point's sequences
//   are contiguous (inf_seq), each sequence's child decision points are
//   contiguous (seq_child) and each level is one range of both.
// * the payoff tensor as a CSR over the player's sequences: one entry per
//   terminal with a nonzero payoff for the player, holding pi_c(z) payoff(z)
//   (FP32 and FP64) and the other players' sequences at z (cols, n-1 per
//   entry, in player order).
//
// Passes per player (a level per launch, so the level barrier is the launch
// boundary and no kernel waits on another; the small top levels of a player
// are one launch of one CTA, a block barrier between levels):
//   rows   u[s] = sum_e val[e] prod_k x_k[col_k[e]]      thread per sequence
//          and, in the same kernel, the average update xbar += t^gamma x
//          (x = 0 adds nothing: skipped)
//   up     level by level, deepest first: np_up_step      thread per decision point
//   down   level by level, from the top: x = x[p_j] b      thread per decision point
// The kernels are launched with programmatic dependent launch (np_enter).
// Iterations are captured as CUDA graphs; the parameters of iteration t come
// from a table that a kernel fills from a device counter at the graph's start.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cfr_nplayer.h"
#include "kernels.cuh"

using namespace cfrb;

namespace {

constexpr int kMaxP = CFRN_MAX_PLAYERS;
constexpr int kThreadsN = 256;
constexpr int kLongRow = 32;    // tensor rows of this many entries or more are summed by a warp
constexpr int kWideKids = 16;   // levels with this many child decision points per sequence go one warp per point

thread_local std::string g_nerr;

int nfail(int status, const std::string &m) {
    g_nerr = m;
    return status;
}

// ---------------------------------------------------------------------------
// host compile
// ---------------------------------------------------------------------------
struct NPlayerHost {
    int32_t J = 0, S = 0;                 // decision points; non-empty sequences
    std::vector<int32_t> inf_seq;         // [J + 1] first sequence of each decision point
    std::vector<int32_t> seq_child;       // [S + 2] first child decision point of each sequence
    std::vector<int32_t> inf_par;         // [J] parent sequence p_j
    std::vector<int32_t> lvl;             // [L + 1] decision points of each level
    std::vector<int32_t> caller_inf;      // [J] caller infoset id of each decision point
    std::vector<int32_t> seq_of_caller;   // [S + 1] sequence of each caller sequence (0 = empty)
    std::vector<int32_t> m_ptr;           // [S + 2]
    std::vector<int32_t> m_col;           // [nnz * (n - 1)]
    std::vector<float> m_val;
    std::vector<double> m_val64;
};

struct NGameHost {
    int n = 0;
    int64_t nodes = 0;
    NPlayerHost pl[kMaxP];
};

std::string at(int64_t i) { return " at node " + std::to_string(i); }

int compile_nplayer(const cfrn_tree_desc &t, NGameHost *g) {
    const int64_t N = t.n_nodes;
    const int n = t.n_players;
    if (n < 2 || n > kMaxP) return nfail(CFR_ERR_INVALID, "n_players must be 2.." + std::to_string(kMaxP));
    if (N < 1) return nfail(CFR_ERR_INVALID, "empty tree");
    if (N >= INT32_MAX) return nfail(CFR_ERR_INVALID, "tree too large for 32-bit indices");
    if (!t.parent || !t.kind || !t.actor || !t.infoset || !t.action || !t.chance_prob || !t.payoff)
        return nfail(CFR_ERR_ARG, "NULL array in the tree");
    if (t.parent[0] != -1) return nfail(CFR_ERR_INVALID, "node 0 must be the root (parent -1)");
    g->n = n;
    g->nodes = N;
    // children per node, action-index checks, infoset sizes
    std::vector<int32_t> nch(N, 0);
    std::vector<uint8_t> seen;   // per child slot
    int32_t J[kMaxP] = {0};
    for (int64_t i = 0; i < N; i++) {
        const int k = t.kind[i];
        if (k < 0 || k > 2) return nfail(CFR_ERR_INVALID, "bad node kind" + at(i));
        if (k == CFRN_DECISION) {
            const int a = t.actor[i];
            if (a < 0 || a >= n) return nfail(CFR_ERR_INVALID, "bad actor" + at(i));
            if (t.infoset[i] < 0) return nfail(CFR_ERR_INVALID, "negative infoset id" + at(i));
            J[a] = std::max(J[a], t.infoset[i] + 1);
        }
        if (i > 0) {
            const int64_t q = t.parent[i];
            if (q < 0 || q >= i) return nfail(CFR_ERR_INVALID, "parent must precede child" + at(i));
            if (t.kind[q] == CFRN_TERMINAL) return nfail(CFR_ERR_INVALID, "terminal with children" + at(q));
            nch[q]++;
        }
    }
    // action indices 0..nch-1 exactly once per parent
    {
        std::vector<int64_t> first(N + 1, 0);
        for (int64_t i = 0; i < N; i++) first[i + 1] = first[i] + nch[i];
        seen.assign(first[N], 0);
        for (int64_t i = 1; i < N; i++) {
            const int64_t q = t.parent[i];
            const int32_t a = t.action[i];
            if (a < 0 || a >= nch[q]) return nfail(CFR_ERR_INVALID, "action index out of range" + at(i));
            if (seen[first[q] + a]) return nfail(CFR_ERR_INVALID, "duplicate action index" + at(i));
            seen[first[q] + a] = 1;
        }
    }
    std::vector<double> psum(N, 0.0);
    for (int64_t i = 1; i < N; i++)
        if (t.kind[t.parent[i]] == CFRN_CHANCE) {
            const double p = t.chance_prob[i];
            if (!(p >= 0.0 && p <= 1.0)) return nfail(CFR_ERR_INVALID, "chance probability outside [0, 1]" + at(i));
            psum[t.parent[i]] += p;
        }
    for (int64_t i = 0; i < N; i++) {
        if (t.kind[i] != CFRN_TERMINAL && nch[i] == 0) return nfail(CFR_ERR_INVALID, "non-terminal leaf" + at(i));
        if (t.kind[i] == CFRN_CHANCE && std::fabs(psum[i] - 1.0) > 1e-9)
            return nfail(CFR_ERR_INVALID, "chance probabilities do not sum to 1" + at(i));
    }
    // actions per infoset (every node of an infoset has the same count)
    std::vector<int32_t> nact[kMaxP], coff[kMaxP];
    for (int p = 0; p < n; p++) nact[p].assign(J[p], -1);
    for (int64_t i = 0; i < N; i++)
        if (t.kind[i] == CFRN_DECISION) {
            int32_t &na = nact[t.actor[i]][t.infoset[i]];
            if (na >= 0 && na != nch[i]) return nfail(CFR_ERR_INVALID, "infoset action counts differ" + at(i));
            na = nch[i];
        }
    int32_t Sc[kMaxP];
    for (int p = 0; p < n; p++) {
        coff[p].assign(J[p], 0);
        int64_t s = 1;
        for (int32_t j = 0; j < J[p]; j++) {
            if (nact[p][j] < 0) return nfail(CFR_ERR_INVALID, "player " + std::to_string(p) + ": infoset id " +
                                                                  std::to_string(j) + " has no node (ids must be dense)");
            coff[p][j] = (int32_t)s;
            s += nact[p][j];
        }
        if (s >= INT32_MAX) return nfail(CFR_ERR_INVALID, "too many sequences");
        Sc[p] = (int32_t)(s - 1);
    }
    // each node's current caller sequence of every player, chance reach,
    // parent caller sequence and level of every infoset (perfect recall)
    std::vector<int32_t> seq((size_t)N * n, 0);
    std::vector<double> reach(N, 1.0);
    std::vector<int32_t> ipar[kMaxP], ilev[kMaxP], iown[kMaxP];
    for (int p = 0; p < n; p++) {
        ipar[p].assign(J[p], -1);
        ilev[p].assign(J[p], -1);
    }
    // decision point owning each caller sequence (for levels)
    for (int p = 0; p < n; p++) {
        iown[p].assign((size_t)Sc[p] + 1, -1);
        for (int32_t j = 0; j < J[p]; j++)
            for (int32_t a = 0; a < nact[p][j]; a++) iown[p][coff[p][j] + a] = j;
    }
    for (int64_t i = 0; i < N; i++) {
        if (i > 0) {
            const int64_t q = t.parent[i];
            std::memcpy(&seq[(size_t)i * n], &seq[(size_t)q * n], sizeof(int32_t) * n);
            reach[i] = reach[q];
            if (t.kind[q] == CFRN_DECISION) seq[(size_t)i * n + t.actor[q]] = coff[t.actor[q]][t.infoset[q]] + t.action[i];
            else if (t.kind[q] == CFRN_CHANCE) reach[i] *= t.chance_prob[i];
        }
        if (t.kind[i] == CFRN_DECISION) {
            const int p = t.actor[i];
            const int32_t j = t.infoset[i], s = seq[(size_t)i * n + p];
            if (ipar[p][j] < 0) {
                ipar[p][j] = s;
                ilev[p][j] = s == 0 ? 0 : ilev[p][iown[p][s]] + 1;
            } else if (ipar[p][j] != s) {
                return nfail(CFR_ERR_INVALID, "imperfect recall: infoset " + std::to_string(j) + " of player " +
                                                  std::to_string(p) + " is reached through different own histories" + at(i));
            }
        }
    }
    // per player: level-by-level numbering
    for (int p = 0; p < n; p++) {
        NPlayerHost &P = g->pl[p];
        P.J = J[p];
        P.S = Sc[p];
        int L = 0;
        for (int32_t j = 0; j < J[p]; j++) L = std::max(L, ilev[p][j] + 1);
        std::vector<std::vector<int32_t>> bylev(L);
        for (int32_t j = 0; j < J[p]; j++) bylev[ilev[p][j]].push_back(j);
        P.seq_of_caller.assign((size_t)Sc[p] + 1, 0);
        P.caller_inf.clear();
        P.inf_seq.assign(1, 1);
        P.inf_par.clear();
        P.lvl.assign(1, 0);
        int32_t snext = 1;
        for (int l = 0; l < L; l++) {
            std::vector<int32_t> &v = bylev[l];
            // by parent sequence (already numbered: one level up), then caller id
            std::sort(v.begin(), v.end(), [&](int32_t a, int32_t b) {
                const int32_t pa = P.seq_of_caller[ipar[p][a]], pb = P.seq_of_caller[ipar[p][b]];
                return pa != pb ? pa < pb : a < b;
            });
            for (int32_t j : v) {
                P.caller_inf.push_back(j);
                P.inf_par.push_back(P.seq_of_caller[ipar[p][j]]);
                for (int32_t a = 0; a < nact[p][j]; a++) P.seq_of_caller[coff[p][j] + a] = snext + a;
                snext += nact[p][j];
                P.inf_seq.push_back(snext);
            }
            P.lvl.push_back((int32_t)P.caller_inf.size());
        }
        // child decision points of each sequence: contiguous, in sequence order
        P.seq_child.assign((size_t)P.S + 2, 0);
        for (int32_t j = 0; j < P.J; j++) P.seq_child[P.inf_par[j] + 1]++;
        for (int64_t s = 0; s < (int64_t)P.S + 1; s++) P.seq_child[s + 1] += P.seq_child[s];
        // (the numbering puts them in that order: check it)
        for (int32_t j = 1; j < P.J; j++)
            if (P.inf_par[j] < P.inf_par[j - 1]) return nfail(CFR_ERR_INVALID, "internal: child order");
    }
    // payoff tensors: one CSR per player over its sequences
    std::vector<int64_t> term;
    for (int64_t i = 0; i < N; i++)
        if (t.kind[i] == CFRN_TERMINAL) term.push_back(i);
    for (int p = 0; p < n; p++) {
        NPlayerHost &P = g->pl[p];
        std::vector<int32_t> cnt((size_t)P.S + 2, 0);
        for (int64_t z : term)
            if (t.payoff[(size_t)z * n + p] != 0.0 && reach[z] != 0.0)
                cnt[P.seq_of_caller[seq[(size_t)z * n + p]] + 1]++;
        for (int64_t s = 0; s < (int64_t)P.S + 1; s++) cnt[s + 1] += cnt[s];
        P.m_ptr = cnt;
        const int64_t nnz = cnt[P.S + 1];
        if (nnz * (n - 1) >= INT32_MAX) return nfail(CFR_ERR_INVALID, "payoff tensor too large");
        P.m_col.assign((size_t)nnz * (n - 1), 0);
        P.m_val.assign(nnz, 0.f);
        P.m_val64.assign(nnz, 0.0);
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t z : term) {
            const double v = t.payoff[(size_t)z * n + p] * reach[z];
            if (t.payoff[(size_t)z * n + p] == 0.0 || reach[z] == 0.0) continue;
            const int32_t e = fill[P.seq_of_caller[seq[(size_t)z * n + p]]]++;
            P.m_val64[e] = v;
            P.m_val[e] = (float)v;
            int c = 0;
            for (int k = 0; k < n; k++)
                if (k != p) P.m_col[(size_t)e * (n - 1) + c++] = g->pl[k].seq_of_caller[seq[(size_t)z * n + k]];
        }
    }
    return CFR_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// device passes
// ---------------------------------------------------------------------------
namespace {

// Programmatic dependent launch: each of an iteration's kernels is launched
// so that it may be scheduled as soon as the previous one completes, before
// that one's memory flush; it waits, first thing, until the previous
// kernel's writes are visible.  The previous kernel does not trigger its
// dependents early: the level grids run several waves, and CTAs of the next
// kernel resident early would take SM slots from the current one's later
// waves (measured slower).
__device__ __forceinline__ void np_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

struct NX {
    const float *x[kMaxP - 1];      // the other players' x, in player order
};
struct NX64 {
    const double *x[kMaxP - 1];
};

// u[s] = sum_e val[e] * prod_k x_k[col_k[e]] for the player's sequences s
// (the payoff tensor contracted with the other players' strategies, Sec. 2.1):
// one thread per sequence, each product taken left to right from val in
// player order and the products added in entry (terminal) order, so the result
// does not depend on the launch shape.  NO: the other players' count.
//
// With `xbar`, the same thread then does the player's average update for its
// sequence, xbar += t^gamma x (x, the player's own strategy, is the one it
// plays this iteration: its bottom-up pass, which comes next, does not change
// it); a sequence with x = 0 adds nothing and is skipped.
//
// R entries at a time: their values and columns are loaded together, then
// their gathers of x, then the products are added in entry order as before
// (R = 4 for players whose rows average kRowBatch entries or more, in games
// of at most kRowBatchMaxOthers + 1 players; shorter rows lose more to the
// padding than they gain, and with more players the batch's gathers take
// too many registers: 8 players went from 491 to 542 us per iteration).
constexpr int kRowBatch = 4;
constexpr int kRowBatchMaxOthers = 4;
template <int NO, int R>
__global__ void __launch_bounds__(kThreadsN) k_np_rows(const int32_t *__restrict__ m_ptr, const int32_t *__restrict__ m_col,
                                                       const float *__restrict__ m_val, NX xs, int S1,
                                                       float *__restrict__ u, float2 *__restrict__ xbar,
                                                       const float *__restrict__ xown,
                                                       const ItemParams *__restrict__ par, int slot, int long_min) {
    np_enter();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S1) return;
    const int e0 = m_ptr[s], e1 = m_ptr[s + 1];
    if (e1 - e0 < long_min) {   // longer rows: k_np_rows_long
        float acc = 0.f;
        for (int e = e0; e < e1; e += R) {
            float v[R];
            int32_t cc[R][NO];
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int64_t er = min(e + r, e1 - 1);   // past the row: a repeat, not added
                v[r] = m_val[er];
#pragma unroll
                for (int k = 0; k < NO; k++) cc[r][k] = m_col[er * NO + k];
            }
            float xv[R][NO];
#pragma unroll
            for (int r = 0; r < R; r++)
#pragma unroll
                for (int k = 0; k < NO; k++) xv[r][k] = __ldg(xs.x[k] + cc[r][k]);
#pragma unroll
            for (int r = 0; r < R; r++)
                if (e + r < e1) {
                    float pv = v[r];
#pragma unroll
                    for (int k = 0; k < NO; k++) pv = __fmul_rn(pv, xv[r][k]);
                    acc = __fadd_rn(acc, pv);
                }
        }
        u[s] = acc;
    }
    if (xbar) {
        const float xv = xown[s];
        if (xv != 0.f) xbar[s] = ff_add(xbar[s], ff_mul_f(par[slot].w, xv));
    }
}

// G lanes per row for players with long rows: lane k takes the entries k,
// k+G, ... in order, a fixed butterfly over the G lanes adds their sums, and
// lane 0 stores u and does the average update.  G is taken from the game
// alone (row_lanes below), so the order depends only on the game.  A group's
// lanes are all in the same warp and share its row, so a group is active or
// exits as a whole.
template <int NO, int G>
__global__ void __launch_bounds__(kThreadsN) k_np_rows_g(const int32_t *__restrict__ m_ptr,
                                                         const int32_t *__restrict__ m_col,
                                                         const float *__restrict__ m_val, NX xs, int S1,
                                                         float *__restrict__ u, float2 *__restrict__ xbar,
                                                         const float *__restrict__ xown,
                                                         const ItemParams *__restrict__ par, int slot, int long_min) {
    np_enter();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = tid / G;
    if (s >= S1) return;
    const int lane = threadIdx.x & (G - 1);
    const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << ((threadIdx.x & 31) & ~(G - 1));
    const int e0 = m_ptr[s], e1 = m_ptr[s + 1];
    if (e1 - e0 < long_min) {   // longer rows: k_np_rows_long
        float acc = 0.f;
        for (int e = e0 + lane; e < e1; e += G) {
            float v = m_val[e];
            const int32_t *c = m_col + (int64_t)e * NO;
#pragma unroll
            for (int k = 0; k < NO; k++) v = __fmul_rn(v, __ldg(xs.x[k] + c[k]));
            acc = __fadd_rn(acc, v);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(gmask, acc, o, G));
        if (lane == 0) u[s] = acc;
    }
    if (xbar && lane == 0) {
        const float xv = xown[s];
        if (xv != 0.f) xbar[s] = ff_add(xbar[s], ff_mul_f(par[slot].w, xv));
    }
}

// Rows of kLongRow or more entries (games with many players between a
// player's decisions), one warp per row: lane k takes the entries k, k+32,
// ... in order, then a fixed butterfly adds the lanes' sums.  long_rows: the
// rows' sequences, listed at load.
template <int NO>
__global__ void __launch_bounds__(kThreadsN) k_np_rows_long(const int32_t *__restrict__ m_ptr,
                                                            const int32_t *__restrict__ m_col,
                                                            const float *__restrict__ m_val, NX xs,
                                                            const int32_t *__restrict__ long_rows, int n_long,
                                                            float *__restrict__ u) {
    np_enter();
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= n_long) return;   // whole warps
    const int s = long_rows[w];
    const int e0 = m_ptr[s], e1 = m_ptr[s + 1];
    float acc = 0.f;
    for (int e = e0 + lane; e < e1; e += 32) {
        float v = m_val[e];
        const int32_t *c = m_col + (int64_t)e * NO;
#pragma unroll
        for (int k = 0; k < NO; k++) v = __fmul_rn(v, __ldg(xs.x[k] + c[k]));
        acc = __fadd_rn(acc, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (lane == 0) u[s] = acc;
}

// the same in FP64 for the best responses (the others' normalised averages)
template <int NO>
__global__ void __launch_bounds__(kThreadsN) k_np_rows64(const int32_t *__restrict__ m_ptr, const int32_t *__restrict__ m_col,
                                                         const double *__restrict__ m_val, NX64 xs, int S1,
                                                         double *__restrict__ u) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S1) return;
    const int e0 = m_ptr[s], e1 = m_ptr[s + 1];
    double acc = 0.0;
    for (int e = e0; e < e1; e++) {
        double v = m_val[e];
        const int32_t *c = m_col + (int64_t)e * NO;
#pragma unroll
        for (int k = 0; k < NO; k++) v *= __ldg(xs.x[k] + c[k]);
        acc += v;
    }
    u[s] = acc;
}

// One level of ObserveUtility + NextStrategy (Alg. 1/2 with the variant's
// post-op): the two-player path's per-infoset step (up_infoset_cfr), for a
// decision point of at most kNpA actions with its loads issued together: u, b, r and the child pointers of all its sequences at
// once, then the children's ev (contiguous across its sequences) eight at a
// time, each added to its own sequence's V in child order.  The arithmetic is
// up_infoset_cfr's, in the same order (V = u + children left to right;
// ev = fma chain over the actions; r, the post-op, regret matching), so the
// results are identical.  Wider decision points take up_infoset_cfr.
constexpr int kNpA = 4;
constexpr int kNpKids = 16;   // children's ev loads in flight (8: slower on wide top levels; 32: spills)
// LEAF: a player's deepest level, whose sequences have no child decision
// points (their child ranges are not read).
template <int VAR, bool LEAF = false>
__device__ __forceinline__ void np_up_step(const DevPlayer &P, int j, const ItemParams &ip) {
    const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
    const int na = s1 - s0;
    if (na > kNpA) {
        up_infoset_cfr(P, j, VAR, ip);
        return;
    }
    float uv[kNpA], bv[kNpA];
    float2 rv[kNpA];
    int cb[kNpA + 1];
#pragma unroll
    for (int a = 0; a < kNpA; a++)
        if (a < na) {
            uv[a] = P.u[s0 + a];
            bv[a] = P.b[s0 + a];
            rv[a] = P.r[s0 + a];
        }
#pragma unroll
    for (int a = 0; a <= kNpA; a++)
        if (a <= na) cb[a] = LEAF ? 0 : P.seq_child[s0 + a];
    // the children's ev, kNpKids loads in flight; child c belongs to the
    // action a with cb[a] <= c < cb[a+1]
    int c1 = cb[0];   // cb[na], with static indices only (cb stays in registers)
#pragma unroll
    for (int a = 1; a <= kNpA; a++)
        if (a == na) c1 = cb[a];
    const int c0 = cb[0];
    for (int c = c0; c < c1; c += kNpKids) {
        float e[kNpKids];
#pragma unroll
        for (int k = 0; k < kNpKids; k++) e[k] = __ldcg(&P.ev[min(c + k, c1 - 1)]);
#pragma unroll
        for (int k = 0; k < kNpKids; k++) {
            const int cc = c + k;
            if (cc < c1) {
#pragma unroll
                for (int a = 0; a < kNpA; a++)
                    if (a < na && cc >= cb[a] && cc < cb[a + 1]) uv[a] += e[k];
            }
        }
    }
    float ev = 0.f;
#pragma unroll
    for (int a = 0; a < kNpA; a++)
        if (a < na) ev = fmaf(bv[a], uv[a], ev);
    P.ev[j] = ev;
    const bool pred = predictive(VAR);
    float pos = 0.f, q[kNpA];
#pragma unroll
    for (int a = 0; a < kNpA; a++)
        if (a < na) {
            const float d = uv[a] - ev;
            float2 r = ff_add_f(rv[a], d);
            r = post_op_v<VAR>(r, ip.fpos, ip.fneg);
            P.r[s0 + a] = r;
            const float rr = pred ? r.x + d : r.x;
            q[a] = rr > 0.f ? rr : 0.f;
            pos += q[a];
        }
    const RmNorm nrm = rm_norm(pos);
    const float uni = uniform_prob(na);
#pragma unroll
    for (int a = 0; a < kNpA; a++)
        if (a < na) P.b[s0 + a] = pos > 0.f ? rm_prob(q[a], nrm) : uni;
}

template <int VAR, bool LEAF>
__global__ void __launch_bounds__(kThreadsN) k_np_up2(DevPlayer P, int j0, int j1, const ItemParams *__restrict__ par,
                                                      int slot) {
    np_enter();
    const int j = j0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= j1) return;
    const ItemParams ip = par[slot];
    np_up_step<VAR, LEAF>(P, j, ip);
}

// A level whose sequences have many child decision points (kWideKids or
// more on average), one warp per decision point: for each of its sequences
// lane k sums the children k, k+32, ... in order, a fixed butterfly adds the
// lanes' sums, lane 0 adds them to u; then lane 0 takes the decision point's
// step with an empty child map (P's seq_child all zero), so V = that u.
template <int VAR>
__global__ void __launch_bounds__(kThreadsN) k_np_up_wide(DevPlayer P, const int32_t *__restrict__ seq_child, int j0,
                                                          int j1, const ItemParams *__restrict__ par, int slot) {
    np_enter();
    const int j = j0 + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (j >= j1) return;   // whole warps
    const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
    for (int s = s0; s < s1; s++) {
        const int c0 = seq_child[s], c1 = seq_child[s + 1];
        float part = 0.f;
        for (int c = c0 + lane; c < c1; c += 32) part = __fadd_rn(part, __ldcg(&P.ev[c]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, o));
        if (lane == 0) P.u[s] = __fadd_rn(P.u[s], part);
    }
    if (lane == 0) {
        const ItemParams ip = par[slot];
        np_up_step<VAR>(P, j, ip);
    }
}

// The small top levels of a player (levels 0 .. m-1, each at most kTopLevel
// decision points) in one launch of one CTA: the levels in order, a block
// barrier between them.  Values of the level below another thread wrote are
// read through L2 (ld.cg: the writes of a CTA's threads are visible to it
// after the barrier; L1 could hold a stale line next to them).  A level of
// more decision points gets a launch of its own: one SM's scattered loads of
// its children's ev (a sector each) would take longer than a launch boundary
// (a three-player game's top launch of 4, 64 and 1,119 points took 24 us).
constexpr int kTopLevel = 256;
constexpr int kTopThreads = 1024;
constexpr int kMaxLevels = 32;
struct NLv {
    int32_t j[kMaxLevels + 1];
};
template <int VAR>
__global__ void __launch_bounds__(kTopThreads) k_np_up_top(DevPlayer P, NLv lv, int m,
                                                           const ItemParams *__restrict__ par, int slot) {
    np_enter();
    const ItemParams ip = par[slot];
    for (int l = m - 1; l >= 0; l--) {
        for (int j = lv.j[l] + threadIdx.x; j < lv.j[l + 1]; j += blockDim.x) np_up_step<VAR>(P, j, ip);
        __syncthreads();
    }
}
__global__ void __launch_bounds__(kTopThreads) k_np_down_top(const int32_t *__restrict__ inf_seq,
                                                             const int32_t *__restrict__ inf_par,
                                                             const float *__restrict__ b, float *__restrict__ x, NLv lv,
                                                             int m) {
    np_enter();
    for (int l = 0; l < m; l++) {
        for (int j = lv.j[l] + threadIdx.x; j < lv.j[l + 1]; j += blockDim.x) {
            const float xp = __ldcg(&x[inf_par[j]]);
            for (int s = inf_seq[j]; s < inf_seq[j + 1]; s++) x[s] = __fmul_rn(xp, b[s]);
        }
        __syncthreads();
    }
}

// one level of the sequence form, top-down: x[(j,a)] = x[p_j] b_j[a]
__global__ void __launch_bounds__(kThreadsN) k_np_down(const int32_t *__restrict__ inf_seq,
                                                       const int32_t *__restrict__ inf_par,
                                                       const float *__restrict__ b, float *__restrict__ x, int j0,
                                                       int j1) {
    np_enter();
    const int j = j0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= j1) return;
    const float xp = x[inf_par[j]];
    for (int s = inf_seq[j]; s < inf_seq[j + 1]; s++) x[s] = __fmul_rn(xp, b[s]);
}

// All levels of the sequence form in one launch: a decision point j walks
// its ancestor sequences p_j, p_(owner of p_j), ... up to the empty sequence
// through seq_up (the parent sequence of each sequence's decision point),
// then multiplies their b from the top down, which is the product the
// level-by-level pass forms, rounding for rounding:
// x[p_j] = ((1 * b[top]) * ...) * b[p_j], then x[(j,a)] = x[p_j] b_j[a].
// The walk is a chain of dependent loads, so each thread takes U decision
// points (j, j + T, ..., T the grid's threads) and interleaves their walks;
// D bounds a walk's length (a player's levels minus one).  No thread waits
// on another.
template <int D, int U>
__global__ void __launch_bounds__(kThreadsN) k_np_down_walk(const int32_t *__restrict__ inf_seq,
                                                            const int32_t *__restrict__ inf_par,
                                                            const int32_t *__restrict__ seq_up,
                                                            const float *__restrict__ b, float *__restrict__ x, int J) {
    np_enter();
    const int64_t T = (int64_t)gridDim.x * blockDim.x, t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // every walk's first loads, and the b of each point's first kNpA
    // actions, issued together
    int q[U], d[U], s0[U], s1[U];
    float bs[U][kNpA];
#pragma unroll
    for (int u = 0; u < U; u++) {
        const int64_t j = t + u * T;
        const bool in = j < J;
        q[u] = in ? inf_par[j] : 0;
        s0[u] = in ? inf_seq[j] : 0;
        s1[u] = in ? inf_seq[j + 1] : 0;
        d[u] = 0;
    }
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
        for (int a = 0; a < kNpA; a++) bs[u][a] = s0[u] + a < s1[u] ? b[s0[u] + a] : 0.0f;
    float bb[U][D];
#pragma unroll
    for (int k = 0; k < D; k++) {
#pragma unroll
        for (int u = 0; u < U; u++)
            if (q[u] != 0) {
                bb[u][k] = b[q[u]];
                q[u] = seq_up[q[u]];
                d[u] = k + 1;
            }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
        float xp = 1.0f;
#pragma unroll
        for (int k = D - 1; k >= 0; k--)
            if (k < d[u]) xp = __fmul_rn(xp, bb[u][k]);
#pragma unroll
        for (int a = 0; a < kNpA; a++)
            if (s0[u] + a < s1[u]) x[s0[u] + a] = __fmul_rn(xp, bs[u][a]);
        for (int s = s0[u] + kNpA; s < s1[u]; s++) x[s] = __fmul_rn(xp, b[s]);
    }
}
constexpr int kWalk = 16;   // longest walk (players of at most kWalk + 1 levels)

// initial behavioural strategy: uniform at every decision point
__global__ void k_np_uniform(const int32_t *__restrict__ inf_seq, float *__restrict__ b, int J) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const int s0 = inf_seq[j], s1 = inf_seq[j + 1];
    const float p = uniform_prob(s1 - s0);
    for (int s = s0; s < s1; s++) b[s] = p;
}

// parameters of iterations t0+1 .. t0+k (t0 read from the device counter):
// t^gamma; DCFR's t^alpha/(t^alpha+1) and t^beta/(t^beta+1)
__global__ void k_np_params(ItemParams *__restrict__ par, const int32_t *__restrict__ t_dev, int k, int variant,
                            double alpha, double beta, double gamma) {
    np_enter();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= k) return;
    const int32_t t = *t_dev + s + 1;
    const double td = (double)t;
    ItemParams ip;
    ip.t = t;
    ip.active = 1;
    ip.w = ff_from_double(pow(td, gamma));
    if (variant == VAR_DCFR) {
        const double ta = pow(td, alpha), tb = pow(td, beta);
        ip.fpos = ff_from_double(ta / (ta + 1.0));
        ip.fneg = ff_from_double(tb / (tb + 1.0));
    } else {
        ip.fpos = make_float2(1.f, 0.f);
        ip.fneg = make_float2(1.f, 0.f);
    }
    par[s] = ip;
}
__global__ void k_np_tick(int32_t *t_dev, int k) {
    np_enter();
    *t_dev += k;
}

// the player's normalised average xbar / xbar[empty] (the current x before
// any iteration), FP64
__global__ void __launch_bounds__(kThreadsN) k_np_avgnorm(const float2 *__restrict__ xbar, const float *__restrict__ x,
                                                          double *__restrict__ x64, int S1) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S1) return;
    const double d0 = (double)xbar[0].x + (double)xbar[0].y;
    x64[s] = d0 > 0.0 ? ((double)xbar[s].x + (double)xbar[s].y) / d0 : (double)x[s];
}

// one level of the best response: ev = max_a V
__global__ void __launch_bounds__(kThreadsN) k_np_br(DevPlayer P, int j0, int j1) {
    const int j = j0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j < j1) up_infoset_br(P, j);
}

// out[0] = <x, u> (the player's value against the others), out[1] = its best
// response's value u[empty] + sum of the top decision points' ev.  One CTA:
// strided partial sums per thread, then a fixed tree, so the order is fixed.
__global__ void __launch_bounds__(kThreadsN) k_np_value(const double *__restrict__ x64, const double *__restrict__ u64,
                                                        int S1, const int32_t *__restrict__ seq_child,
                                                        const double *__restrict__ ev64, double *__restrict__ out) {
    __shared__ double part[kThreadsN];
    double acc = 0.0;
    for (int s = threadIdx.x; s < S1; s += blockDim.x) acc += x64[s] * u64[s];
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = part[0];
        double br = u64[0];
        for (int c = seq_child[0]; c < seq_child[1]; c++) br += ev64[c];
        out[1] = br;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
namespace {

constexpr int kParamCap = 1024;   // iterations per graph at most (parameter table)

struct NDev {
    int32_t J = 0, S = 0, L = 0;
    int64_t nnz = 0;
    std::vector<int32_t> lvl;     // host copy: decision points of each level
    int mtop = 0;                 // top levels (from level 0) of at most kTopLevel decision points each
    int32_t *inf_seq = nullptr, *seq_child = nullptr, *inf_par = nullptr, *m_ptr = nullptr, *m_col = nullptr;
    float *m_val = nullptr;
    double *m_val64 = nullptr;
    float2 *r = nullptr, *xbar = nullptr;
    float *b = nullptr, *x = nullptr, *u = nullptr, *ev = nullptr, *uq = nullptr;
    double *u64 = nullptr, *ev64 = nullptr, *x64 = nullptr;
    int32_t *nokids = nullptr;    // [S + 2] zeros: an empty child map (wide levels' step)
    int32_t *seq_up = nullptr;    // [S + 1] parent sequence of each sequence's decision point (top-down walk)
    bool walk = false;            // top-down in one walking launch (2 to kWalk + 1 levels)
    int32_t *long_rows = nullptr; // sequences whose tensor rows have kLongRow or more entries
    int n_long = 0;
    bool row_batch = false;       // rows k_np_rows takes average kRowBatch entries or more
    int row_lanes = 1;            // lanes per row (4, 8, 16: k_np_rows_g)
    std::vector<uint8_t> wide;    // per level: kWideKids or more child decision points per sequence
    DevPlayer dp{};
    DevPlayer dp_nokids{};        // dp with the empty child map
};

unsigned blocks(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kThreadsN - 1) / kThreadsN); }

}  // namespace

struct cfrn_ctx {
    int n = 0;
    cudaStream_t stream = nullptr;
    NDev P[kMaxP];
    NGameHost host;
    ItemParams *par = nullptr;
    int32_t *t_dev = nullptr;
    double *out = nullptr;              // [2 * kMaxP] values and best responses
    int64_t t = 0;
    int graph_k = 64;
    cudaGraphExec_t graph = nullptr;
    int g_variant = -1, g_alt = -1, g_k = 0;
    double g_a = 0, g_b = 0, g_g = 0;
    int sms = 148;                      // SMs of the device (level launches spread over them)
    int64_t launches = 0;               // kernels run (graph replays count theirs)
    int64_t graph_kernels = 0;          // kernels in the current graph
    bool capturing = false;
    bool own_stream = false;
    int64_t captured = 0;
    std::vector<void *> allocs;
};

namespace {

#define NCU(call)                                                                        \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return nfail(CFR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
int dalloc(cfrn_ctx *c, T **p, int64_t n) {
    *p = nullptr;
    void *q = nullptr;
    NCU(cudaMalloc(&q, (size_t)std::max<int64_t>(n, 1) * sizeof(T)));
    c->allocs.push_back(q);
    *p = (T *)q;
    return CFR_OK;
}
template <class T>
int dput(cfrn_ctx *c, T **p, const std::vector<T> &v) {
    int rc = dalloc(c, p, (int64_t)v.size());
    if (rc) return rc;
    if (!v.empty()) NCU(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return CFR_OK;
}

// launch a pass kernel with programmatic dependent launch (np_enter)
template <class... P, class... A>
cudaError_t np_launch_b(void (*fn)(P...), unsigned grid, unsigned block, cudaStream_t st, A &&...a) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, std::forward<A>(a)...);
}
template <class... P, class... A>
cudaError_t np_launch(void (*fn)(P...), unsigned grid, cudaStream_t st, A &&...a) {
    return np_launch_b(fn, grid, (unsigned)kThreadsN, st, std::forward<A>(a)...);
}

void counted(cfrn_ctx *c, int k = 1) {
    if (c->capturing) c->captured += k;
    else c->launches += k;
}

// the tensor rows of player i into `out`; slot >= 0: also the player's
// average update with the parameters of that slot
// Lanes per row for a player's rows (nnz entries over rows rows, the long
// rows left out), from per-player timings of the 3- to 8-player games: about
// two entries per lane (one thread per row below 8 entries: there more
// lanes only add shuffles and threads), and 16 lanes for players of at most
// kFewRows rows, whose launches are too small to fill the device otherwise.
constexpr int64_t kFewRows = 2048;
int row_lanes(int64_t nnz, int64_t rows) {
    if (rows <= 0 || nnz < 2 * rows) return 1;
    if (rows <= kFewRows) return 16;
    if (nnz >= 16 * rows) return 8;
    if (nnz >= 8 * rows) return 4;
    return 1;
}

template <int NO>
cudaError_t launch_rows(bool batch, unsigned g, cudaStream_t st, const NDev &P, NX xs, int S1, float *out, float2 *xb,
                        const float *xo, const ItemParams *par, int sl, int lm) {
    const int32_t *mp = P.m_ptr, *mc = P.m_col;
    const float *mv = P.m_val;
    switch (P.row_lanes) {
    case 4: return np_launch(k_np_rows_g<NO, 4>, blocks(4ll * S1), st, mp, mc, mv, xs, S1, out, xb, xo, par, sl, lm);
    case 8: return np_launch(k_np_rows_g<NO, 8>, blocks(8ll * S1), st, mp, mc, mv, xs, S1, out, xb, xo, par, sl, lm);
    case 16: return np_launch(k_np_rows_g<NO, 16>, blocks(16ll * S1), st, mp, mc, mv, xs, S1, out, xb, xo, par, sl, lm);
    default: break;
    }
    if constexpr (NO <= kRowBatchMaxOthers)
        if (batch) return np_launch(k_np_rows<NO, kRowBatch>, g, st, mp, mc, mv, xs, S1, out, xb, xo, par, sl, lm);
    return np_launch(k_np_rows<NO, 1>, g, st, mp, mc, mv, xs, S1, out, xb, xo, par, sl, lm);
}

int rows(cfrn_ctx *c, int i, float *out, int slot = -1) {
    NDev &P = c->P[i];
    NX xs{};
    int k = 0;
    for (int q = 0; q < c->n; q++)
        if (q != i) xs.x[k++] = c->P[q].x;
    const int S1 = P.S + 1;
    const unsigned g = blocks(S1);
    cudaStream_t st = c->stream;
    cudaError_t e = cudaSuccess;
    float2 *xb = slot >= 0 ? P.xbar : nullptr;
    const float *xo = P.x;
    const ItemParams *par = c->par;
    const int sl = slot >= 0 ? slot : 0;
    const int lm = P.n_long > 0 ? kLongRow : INT32_MAX;   // rows left to k_np_rows_long
    const bool rb = P.row_batch;
    switch (c->n - 1) {
    case 1: e = launch_rows<1>(rb, g, st, P, xs, S1, out, xb, xo, par, sl, lm); break;
    case 2: e = launch_rows<2>(rb, g, st, P, xs, S1, out, xb, xo, par, sl, lm); break;
    case 3: e = launch_rows<3>(rb, g, st, P, xs, S1, out, xb, xo, par, sl, lm); break;
    case 4: e = launch_rows<4>(rb, g, st, P, xs, S1, out, xb, xo, par, sl, lm); break;
    case 5: e = launch_rows<5>(rb, g, st, P, xs, S1, out, xb, xo, par, sl, lm); break;
    case 6: e = launch_rows<6>(rb, g, st, P, xs, S1, out, xb, xo, par, sl, lm); break;
    default: e = launch_rows<7>(rb, g, st, P, xs, S1, out, xb, xo, par, sl, lm); break;
    }
    if (e != cudaSuccess) return nfail(CFR_ERR_CUDA, std::string("rows launch: ") + cudaGetErrorString(e));
    counted(c);
    if (P.n_long > 0) {
        const unsigned gl = blocks(32ll * P.n_long);
        const int32_t *lr = P.long_rows;
        const int nl = P.n_long;
        switch (c->n - 1) {
        case 1: e = np_launch(k_np_rows_long<1>, gl, st, P.m_ptr, P.m_col, P.m_val, xs, lr, nl, out); break;
        case 2: e = np_launch(k_np_rows_long<2>, gl, st, P.m_ptr, P.m_col, P.m_val, xs, lr, nl, out); break;
        case 3: e = np_launch(k_np_rows_long<3>, gl, st, P.m_ptr, P.m_col, P.m_val, xs, lr, nl, out); break;
        case 4: e = np_launch(k_np_rows_long<4>, gl, st, P.m_ptr, P.m_col, P.m_val, xs, lr, nl, out); break;
        case 5: e = np_launch(k_np_rows_long<5>, gl, st, P.m_ptr, P.m_col, P.m_val, xs, lr, nl, out); break;
        case 6: e = np_launch(k_np_rows_long<6>, gl, st, P.m_ptr, P.m_col, P.m_val, xs, lr, nl, out); break;
        default: e = np_launch(k_np_rows_long<7>, gl, st, P.m_ptr, P.m_col, P.m_val, xs, lr, nl, out); break;
        }
        if (e != cudaSuccess) return nfail(CFR_ERR_CUDA, std::string("long rows launch: ") + cudaGetErrorString(e));
        counted(c);
    }
    return CFR_OK;
}

int rows64(cfrn_ctx *c, int i) {
    NDev &P = c->P[i];
    NX64 xs{};
    int k = 0;
    for (int q = 0; q < c->n; q++)
        if (q != i) xs.x[k++] = c->P[q].x64;
    const int S1 = P.S + 1;
    const unsigned g = blocks(S1);
    cudaStream_t st = c->stream;
    switch (c->n - 1) {
    case 1: k_np_rows64<1><<<g, kThreadsN, 0, st>>>(P.m_ptr, P.m_col, P.m_val64, xs, S1, P.u64); break;
    case 2: k_np_rows64<2><<<g, kThreadsN, 0, st>>>(P.m_ptr, P.m_col, P.m_val64, xs, S1, P.u64); break;
    case 3: k_np_rows64<3><<<g, kThreadsN, 0, st>>>(P.m_ptr, P.m_col, P.m_val64, xs, S1, P.u64); break;
    case 4: k_np_rows64<4><<<g, kThreadsN, 0, st>>>(P.m_ptr, P.m_col, P.m_val64, xs, S1, P.u64); break;
    case 5: k_np_rows64<5><<<g, kThreadsN, 0, st>>>(P.m_ptr, P.m_col, P.m_val64, xs, S1, P.u64); break;
    case 6: k_np_rows64<6><<<g, kThreadsN, 0, st>>>(P.m_ptr, P.m_col, P.m_val64, xs, S1, P.u64); break;
    default: k_np_rows64<7><<<g, kThreadsN, 0, st>>>(P.m_ptr, P.m_col, P.m_val64, xs, S1, P.u64); break;
    }
    counted(c);
    return CFR_OK;
}

NLv top_levels(const NDev &P) {
    NLv lv{};
    for (int l = 0; l <= P.mtop && l <= kMaxLevels; l++) lv.j[l] = P.lvl[l];
    return lv;
}

template <bool LEAF>
void launch_up2(int variant, unsigned g, unsigned tb, cudaStream_t st, const DevPlayer &dp, int j0, int j1,
                const ItemParams *par, int slot) {
    switch (variant) {
    case VAR_PLUS: np_launch_b(k_np_up2<VAR_PLUS, LEAF>, g, tb, st, dp, j0, j1, par, slot); break;
    case VAR_DCFR: np_launch_b(k_np_up2<VAR_DCFR, LEAF>, g, tb, st, dp, j0, j1, par, slot); break;
    case VAR_PCFR_PLUS: np_launch_b(k_np_up2<VAR_PCFR_PLUS, LEAF>, g, tb, st, dp, j0, j1, par, slot); break;
    case VAR_PCFR: np_launch_b(k_np_up2<VAR_PCFR, LEAF>, g, tb, st, dp, j0, j1, par, slot); break;
    default: np_launch_b(k_np_up2<VAR_CFR, LEAF>, g, tb, st, dp, j0, j1, par, slot); break;
    }
}

void up(cfrn_ctx *c, int i, int variant, int slot) {
    NDev &P = c->P[i];
    const int lo = P.mtop >= 2 ? P.mtop : 0;   // levels below lo: one launch each
    for (int l = P.L - 1; l >= lo; l--) {
        const int j0 = P.lvl[l], j1 = P.lvl[l + 1];
        const ItemParams *par = c->par;
        if (P.wide[l]) {
            const unsigned gw = blocks(32ll * (j1 - j0));
            const int32_t *sc = P.seq_child;
            switch (variant) {
            case VAR_PLUS: np_launch(k_np_up_wide<VAR_PLUS>, gw, c->stream, P.dp_nokids, sc, j0, j1, par, slot); break;
            case VAR_DCFR: np_launch(k_np_up_wide<VAR_DCFR>, gw, c->stream, P.dp_nokids, sc, j0, j1, par, slot); break;
            case VAR_PCFR_PLUS:
                np_launch(k_np_up_wide<VAR_PCFR_PLUS>, gw, c->stream, P.dp_nokids, sc, j0, j1, par, slot);
                break;
            case VAR_PCFR: np_launch(k_np_up_wide<VAR_PCFR>, gw, c->stream, P.dp_nokids, sc, j0, j1, par, slot); break;
            default: np_launch(k_np_up_wide<VAR_CFR>, gw, c->stream, P.dp_nokids, sc, j0, j1, par, slot); break;
            }
            counted(c);
            continue;
        }
        // blocks of 32 to kThreadsN threads, about one per SM when the level
        // is small: its children's ev are scattered loads, and one SM's share
        // of them bounds the launch
        const int64_t n = j1 - j0;
        const unsigned tb =
            (unsigned)std::min<int64_t>(kThreadsN, std::max<int64_t>(32, ((n + c->sms - 1) / c->sms + 31) / 32 * 32));
        const unsigned g = (unsigned)((n + tb - 1) / tb);
        if (l == P.L - 1)
            launch_up2<true>(variant, g, tb, c->stream, P.dp, j0, j1, par, slot);
        else
            launch_up2<false>(variant, g, tb, c->stream, P.dp, j0, j1, par, slot);
        counted(c);
    }
    if (lo > 0) {
        const NLv lv = top_levels(P);
        const int m = P.mtop;
        const ItemParams *par = c->par;
        const unsigned T = kTopThreads;
        switch (variant) {
        case VAR_PLUS: np_launch_b(k_np_up_top<VAR_PLUS>, 1u, T, c->stream, P.dp, lv, m, par, slot); break;
        case VAR_DCFR: np_launch_b(k_np_up_top<VAR_DCFR>, 1u, T, c->stream, P.dp, lv, m, par, slot); break;
        case VAR_PCFR_PLUS: np_launch_b(k_np_up_top<VAR_PCFR_PLUS>, 1u, T, c->stream, P.dp, lv, m, par, slot); break;
        case VAR_PCFR: np_launch_b(k_np_up_top<VAR_PCFR>, 1u, T, c->stream, P.dp, lv, m, par, slot); break;
        default: np_launch_b(k_np_up_top<VAR_CFR>, 1u, T, c->stream, P.dp, lv, m, par, slot); break;
        }
        counted(c);
    }
}

void down(cfrn_ctx *c, int i) {
    NDev &P = c->P[i];
    if (P.walk) {
        const int32_t *is = P.inf_seq, *ip = P.inf_par, *su = P.seq_up;
        const float *b = P.b;
        if (P.L - 1 <= 4)
            np_launch(k_np_down_walk<4, 2>, blocks((P.J + 1) / 2), c->stream, is, ip, su, b, P.x, P.J);
        else if (P.L - 1 <= 8)
            np_launch(k_np_down_walk<8, 2>, blocks((P.J + 1) / 2), c->stream, is, ip, su, b, P.x, P.J);
        else
            np_launch(k_np_down_walk<kWalk, 1>, blocks(P.J), c->stream, is, ip, su, b, P.x, P.J);
        counted(c);
        return;
    }
    const int lo = P.mtop >= 2 ? P.mtop : 0;
    if (lo > 0) {
        np_launch_b(k_np_down_top, 1u, (unsigned)kTopThreads, c->stream, (const int32_t *)P.inf_seq,
                    (const int32_t *)P.inf_par, (const float *)P.b, P.x, top_levels(P), lo);
        counted(c);
    }
    for (int l = lo; l < P.L; l++) {
        const int j0 = P.lvl[l], j1 = P.lvl[l + 1];
        np_launch(k_np_down, blocks(j1 - j0), c->stream, (const int32_t *)P.inf_seq, (const int32_t *)P.inf_par,
                  (const float *)P.b, P.x, j0, j1);
        counted(c);
    }
}

void params(cfrn_ctx *c, int k, int variant, double a, double b, double g) {
    np_launch(k_np_params, blocks(k), c->stream, c->par, (const int32_t *)c->t_dev, k, variant, a, b, g);
    counted(c);
}
void tick(cfrn_ctx *c, int k) {
    np_launch(k_np_tick, 1u, c->stream, c->t_dev, k);
    counted(c);
}

// one iteration (parameters in slot `slot` of the table).  ev: optional
// events around each kind of pass, [4][2 * n] (start, end per player).
int iteration(cfrn_ctx *c, int slot, int variant, bool alternating, cudaEvent_t (*ev)[2 * kMaxP] = nullptr) {
    auto mark = [&](int kind, int i, int end) {
        if (ev) cudaEventRecord(ev[kind][2 * i + end], c->stream);
    };
    if (!alternating)
        for (int i = 0; i < c->n; i++) {
            mark(0, i, 0);
            if (int rc = rows(c, i, c->P[i].u, slot)) return rc;
            mark(0, i, 1);
        }
    for (int i = 0; i < c->n; i++) {
        if (alternating) {
            mark(0, i, 0);
            if (int rc = rows(c, i, c->P[i].u, slot)) return rc;
            mark(0, i, 1);
        }
        mark(1, i, 0);
        up(c, i, variant, slot);
        mark(1, i, 1);
        mark(2, i, 0);
        mark(2, i, 1);
        mark(3, i, 0);
        down(c, i);
        mark(3, i, 1);
    }
    return CFR_OK;
}

int run_block(cfrn_ctx *c, int k, int variant, double a, double b, double g, bool alternating) {
    params(c, k, variant, a, b, g);
    for (int s = 0; s < k; s++)
        if (int rc = iteration(c, s, variant, alternating)) return rc;
    tick(c, k);
    NCU(cudaGetLastError());
    return CFR_OK;
}

int ensure_graph(cfrn_ctx *c, int k, int variant, double a, double b, double g, bool alternating) {
    if (c->graph && c->g_k == k && c->g_variant == variant && c->g_alt == (int)alternating && c->g_a == a &&
        c->g_b == b && c->g_g == g)
        return CFR_OK;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    cudaGraph_t gr = nullptr;
    NCU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    c->captured = 0;
    int rc = run_block(c, k, variant, a, b, g, alternating);
    c->capturing = false;
    cudaError_t e = cudaStreamEndCapture(c->stream, &gr);
    if (rc) {
        if (gr) cudaGraphDestroy(gr);
        return rc;
    }
    if (e != cudaSuccess) return nfail(CFR_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        return nfail(CFR_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    NCU(cudaGraphUpload(c->graph, c->stream));
    c->graph_kernels = c->captured;
    c->g_k = k;
    c->g_variant = variant;
    c->g_alt = (int)alternating;
    c->g_a = a;
    c->g_b = b;
    c->g_g = g;
    return CFR_OK;
}

void free_ctx(cfrn_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (void *p : c->allocs) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int check_player(const cfrn_ctx *c, int p) {
    if (!c) return nfail(CFR_ERR_ARG, "NULL context");
    if (p < 0 || p >= c->n) return nfail(CFR_ERR_ARG, "player outside 0..n-1");
    return CFR_OK;
}

int load(const cfrn_tree_desc *tree, void *stream, cfrn_ctx **out) {
    if (!tree || !out) return nfail(CFR_ERR_ARG, "NULL argument");
    *out = nullptr;
    cfrn_ctx *c = new cfrn_ctx();
    int rc = compile_nplayer(*tree, &c->host);
    auto bail = [&](int r) {
        free_ctx(c);
        return r;
    };
    if (rc) return bail(rc);
    // a stream of its own unless one is given (graphs cannot be captured on
    // the legacy default stream)
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(nfail(CFR_ERR_CUDA, "stream creation failed"));
        c->own_stream = true;
    }
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c->sms < 1)
            return bail(nfail(CFR_ERR_CUDA, "querying the device"));
    }
    c->n = c->host.n;
    std::vector<int32_t> ups[kMaxP];   // host sources of the seq_up uploads, alive until the sync below
    for (int p = 0; p < c->n; p++) {
        NPlayerHost &H = c->host.pl[p];
        NDev &P = c->P[p];
        P.J = H.J;
        P.S = H.S;
        P.L = (int)H.lvl.size() - 1;
        P.lvl = H.lvl;
        P.nnz = (int64_t)H.m_val.size();
        const int64_t S1 = (int64_t)P.S + 1;
        // levels whose sequences have kWideKids or more child decision points
        // on average are worked one warp per decision point
        P.wide.assign(P.L, 0);
        for (int l = 0; l < P.L; l++) {
            const int64_t s0 = H.inf_seq[H.lvl[l]], s1 = H.inf_seq[H.lvl[l + 1]];
            const int64_t kids = (int64_t)H.seq_child[s1] - H.seq_child[s0];
            P.wide[l] = s1 > s0 && kids >= (int64_t)kWideKids * (s1 - s0);
        }
        while (P.mtop < P.L && P.mtop < kMaxLevels && P.lvl[P.mtop + 1] - P.lvl[P.mtop] <= kTopLevel &&
               !P.wide[P.mtop])
            P.mtop++;
        {
            // rows of kLongRow or more entries go to a warp each, when they hold
            // at least a tenth of the player's entries (else one more launch
            // costs more than their serial sums)
            std::vector<int32_t> lr;
            int64_t in_long = 0;
            for (int64_t s = 0; s < S1; s++)
                if (H.m_ptr[s + 1] - H.m_ptr[s] >= kLongRow) {
                    lr.push_back((int32_t)s);
                    in_long += H.m_ptr[s + 1] - H.m_ptr[s];
                }
            if (10 * in_long < (int64_t)H.m_val.size()) lr.clear();
            P.n_long = (int)lr.size();
            const int64_t short_nnz = (int64_t)H.m_val.size() - (lr.empty() ? 0 : in_long);
            P.row_batch = short_nnz >= (int64_t)kRowBatch * (S1 - P.n_long);
            P.row_lanes = row_lanes(short_nnz, S1 - P.n_long);
            if ((rc = dput(c, &P.long_rows, lr)) || (rc = dalloc(c, &P.nokids, S1 + 1))) return bail(rc);
            if (cudaMemsetAsync(P.nokids, 0, (S1 + 1) * sizeof(int32_t), c->stream) != cudaSuccess)
                return bail(nfail(CFR_ERR_CUDA, "initialising the empty child map"));
        }
        // top-down in one walking launch for players of 2 to kWalk + 1 levels
        // (one level: its single launch needs no walk)
        P.walk = P.J > 0 && P.L >= 2 && P.L - 1 <= kWalk;
        if (P.walk) {
            std::vector<int32_t> &up = ups[p];
            up.assign((size_t)S1, 0);
            for (int32_t j = 0; j < P.J; j++)
                for (int32_t s = H.inf_seq[j]; s < H.inf_seq[j + 1]; s++) up[s] = H.inf_par[j];
            if ((rc = dput(c, &P.seq_up, up))) return bail(rc);
        }
        if ((rc = dput(c, &P.inf_seq, H.inf_seq)) || (rc = dput(c, &P.seq_child, H.seq_child)) ||
            (rc = dput(c, &P.inf_par, H.inf_par)) || (rc = dput(c, &P.m_ptr, H.m_ptr)) ||
            (rc = dput(c, &P.m_col, H.m_col)) || (rc = dput(c, &P.m_val, H.m_val)) ||
            (rc = dput(c, &P.m_val64, H.m_val64)) || (rc = dalloc(c, &P.r, S1)) || (rc = dalloc(c, &P.xbar, S1)) ||
            (rc = dalloc(c, &P.b, S1)) || (rc = dalloc(c, &P.x, S1)) || (rc = dalloc(c, &P.u, S1)) ||
            (rc = dalloc(c, &P.uq, S1)) || (rc = dalloc(c, &P.ev, P.J)) || (rc = dalloc(c, &P.u64, S1)) ||
            (rc = dalloc(c, &P.ev64, P.J)) || (rc = dalloc(c, &P.x64, S1)))
            return bail(rc);
        DevPlayer &d = P.dp;
        d.inf_seq = P.inf_seq;
        d.seq_child = P.seq_child;
        d.inf_par = P.inf_par;
        d.r = P.r;
        d.b = P.b;
        d.x = P.x;
        d.xbar = P.xbar;
        d.u = P.u;
        d.ev = P.ev;
        d.u64 = P.u64;
        d.ev64 = P.ev64;
        d.S = (int32_t)S1;
        d.G = 1;
        P.dp_nokids = d;
        P.dp_nokids.seq_child = P.nokids;
        if (cudaMemsetAsync(P.r, 0, S1 * sizeof(float2), c->stream) != cudaSuccess ||
            cudaMemsetAsync(P.xbar, 0, S1 * sizeof(float2), c->stream) != cudaSuccess ||
            cudaMemsetAsync(P.b, 0, S1 * sizeof(float), c->stream) != cudaSuccess ||
            cudaMemsetAsync(P.x, 0, S1 * sizeof(float), c->stream) != cudaSuccess)
            return bail(nfail(CFR_ERR_CUDA, "initialising the state"));
        static const float one = 1.0f;
        if (cudaMemcpyAsync(P.x, &one, sizeof(float), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return bail(nfail(CFR_ERR_CUDA, "initialising x"));
        if (P.J > 0) k_np_uniform<<<blocks(P.J), kThreadsN, 0, c->stream>>>(P.inf_seq, P.b, P.J);
        counted(c);
    }
    if ((rc = dalloc(c, &c->par, kParamCap)) || (rc = dalloc(c, &c->t_dev, 1)) || (rc = dalloc(c, &c->out, 2 * kMaxP)))
        return bail(rc);
    if (cudaMemsetAsync(c->t_dev, 0, sizeof(int32_t), c->stream) != cudaSuccess)
        return bail(nfail(CFR_ERR_CUDA, "initialising t"));
    for (int p = 0; p < c->n; p++) down(c, p);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return bail(nfail(CFR_ERR_CUDA, "initial strategies"));
    // the host copies of the layout are kept for the state read-back
    for (int p = 0; p < c->n; p++) {
        NPlayerHost &H = c->host.pl[p];
        std::vector<int32_t>().swap(H.m_ptr);
        std::vector<int32_t>().swap(H.m_col);
        std::vector<float>().swap(H.m_val);
        std::vector<double>().swap(H.m_val64);
    }
    *out = c;
    return CFR_OK;
}

// caller numbering: caller sequence c (1..S) of player p is sequence
// seq_of_caller[c]; arrays of S entries skip the empty sequence
template <class T, class F>
void to_caller(const NPlayerHost &H, const std::vector<T> &dev, double *dst, bool with_empty, F conv) {
    const int64_t S = H.S;
    if (with_empty) dst[0] = conv(dev[0]);
    for (int64_t k = 1; k <= S; k++) dst[with_empty ? k : k - 1] = conv(dev[H.seq_of_caller[k]]);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int cfrn_load(const cfrn_tree_desc *tree, void *stream, cfrn_ctx **out) { return load(tree, stream, out); }

int cfrn_check_tree(const cfrn_tree_desc *tree, int64_t *sizes) {
    if (!tree) return nfail(CFR_ERR_ARG, "NULL tree");
    NGameHost g;
    if (int rc = compile_nplayer(*tree, &g)) return rc;
    if (sizes)
        for (int p = 0; p < g.n; p++) {
            const NPlayerHost &H = g.pl[p];
            sizes[4 * p + 0] = H.J;
            sizes[4 * p + 1] = H.S;
            sizes[4 * p + 2] = (int64_t)H.lvl.size() - 1;
            sizes[4 * p + 3] = (int64_t)H.m_val.size();
        }
    return CFR_OK;
}

int cfrn_free(cfrn_ctx *ctx) {
    free_ctx(ctx);
    return CFR_OK;
}

const char *cfrn_last_error(void) { return g_nerr.c_str(); }

int cfrn_sizes(const cfrn_ctx *ctx, int player, int64_t *out) {
    if (int rc = check_player(ctx, player)) return rc;
    if (!out) return nfail(CFR_ERR_ARG, "NULL output");
    const NDev &P = ctx->P[player];
    out[0] = P.J;
    out[1] = P.S;
    out[2] = P.L;
    out[3] = P.nnz;
    out[4] = ctx->n;
    out[5] = ctx->t;
    int64_t k = 0;   // kernels of one iteration: every player's rows, bottom-up and top-down launches
    for (int p = 0; p < ctx->n; p++) {
        const NDev &Q = ctx->P[p];
        const int levels = Q.mtop >= 2 ? Q.L - Q.mtop + 1 : Q.L;
        k += 1 + (Q.n_long > 0 ? 1 : 0) + levels + (Q.walk ? 1 : levels);
    }
    out[6] = k;
    return CFR_OK;
}

int cfrn_level_sizes(const cfrn_ctx *ctx, int player, int64_t *out, int cap) {
    if (int rc = check_player(ctx, player)) return rc;
    if (!out || cap < 0) return nfail(CFR_ERR_ARG, "NULL output or negative capacity");
    const NDev &P = ctx->P[player];
    const NPlayerHost &H = ctx->host.pl[player];
    for (int l = 0; l < std::min(P.L, cap); l++) {
        out[2 * l] = P.lvl[l + 1] - P.lvl[l];
        out[2 * l + 1] = (int64_t)H.inf_seq[P.lvl[l + 1]] - H.inf_seq[P.lvl[l]];
    }
    return CFR_OK;
}

int cfrn_set_graph_iterations(cfrn_ctx *ctx, int k) {
    if (!ctx) return nfail(CFR_ERR_ARG, "NULL context");
    if (k < 1 || k > kParamCap) return nfail(CFR_ERR_ARG, "graph iterations must be 1..1024");
    ctx->graph_k = k;
    return CFR_OK;
}

int cfrn_iterate(cfrn_ctx *ctx, int64_t n, int variant, double alpha, double beta, double gamma, int alternating) {
    if (!ctx) return nfail(CFR_ERR_ARG, "NULL context");
    if (n < 0 || variant < 0 || variant > 4) return nfail(CFR_ERR_ARG, "bad iteration count or variant");
    if (ctx->t + n >= INT32_MAX) return nfail(CFR_ERR_ARG, "iteration counter would overflow");
    const bool alt = alternating != 0;
    while (n > 0) {
        const int K = ctx->graph_k;
        if (K > 1 && n >= K) {
            if (int rc = ensure_graph(ctx, K, variant, alpha, beta, gamma, alt)) return rc;
            NCU(cudaGraphLaunch(ctx->graph, ctx->stream));
            ctx->launches += ctx->graph_kernels;
            ctx->t += K;
            n -= K;
        } else {
            const int k = (int)std::min<int64_t>(n, K);
            if (int rc = run_block(ctx, k, variant, alpha, beta, gamma, alt)) return rc;
            ctx->t += k;
            n -= k;
        }
    }
    return CFR_OK;
}

int cfrn_prepare_graph(cfrn_ctx *ctx, int variant, double alpha, double beta, double gamma, int alternating) {
    if (!ctx) return nfail(CFR_ERR_ARG, "NULL context");
    if (variant < 0 || variant > 4) return nfail(CFR_ERR_ARG, "bad variant");
    if (ctx->graph_k < 2) return CFR_OK;   // eager launches: no graph
    return ensure_graph(ctx, ctx->graph_k, variant, alpha, beta, gamma, alternating != 0);
}

int cfrn_sync(cfrn_ctx *ctx) {
    if (!ctx) return nfail(CFR_ERR_ARG, "NULL context");
    NCU(cudaStreamSynchronize(ctx->stream));
    NCU(cudaGetLastError());
    return CFR_OK;
}

int cfrn_get_state(cfrn_ctx *ctx, int player, double *r, double *b, double *xbar, int64_t *t) {
    if (int rc = check_player(ctx, player)) return rc;
    if (int rc = cfrn_sync(ctx)) return rc;
    const NDev &P = ctx->P[player];
    const NPlayerHost &H = ctx->host.pl[player];
    const int64_t S1 = (int64_t)P.S + 1;
    auto ff = [](float2 v) { return (double)v.x + (double)v.y; };
    auto fl = [](float v) { return (double)v; };
    if (r) {
        std::vector<float2> h(S1);
        NCU(cudaMemcpy(h.data(), P.r, S1 * sizeof(float2), cudaMemcpyDeviceToHost));
        to_caller(H, h, r, false, ff);
    }
    if (b) {
        std::vector<float> h(S1);
        NCU(cudaMemcpy(h.data(), P.b, S1 * sizeof(float), cudaMemcpyDeviceToHost));
        to_caller(H, h, b, false, fl);
    }
    if (xbar) {
        std::vector<float2> h(S1);
        NCU(cudaMemcpy(h.data(), P.xbar, S1 * sizeof(float2), cudaMemcpyDeviceToHost));
        to_caller(H, h, xbar, true, ff);
    }
    if (t) *t = ctx->t;
    return CFR_OK;
}

int cfrn_set_state(cfrn_ctx *ctx, int player, const double *r, const double *b, const double *xbar, int64_t t) {
    if (int rc = check_player(ctx, player)) return rc;
    if (t >= INT32_MAX) return nfail(CFR_ERR_ARG, "iteration counter too large");
    if (int rc = cfrn_sync(ctx)) return rc;
    NDev &P = ctx->P[player];
    const NPlayerHost &H = ctx->host.pl[player];
    const int64_t S1 = (int64_t)P.S + 1;
    auto ff = [](double v) {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    };
    if (b) {   // a distribution at every decision point (caller numbering: off_j + a)
        std::vector<int32_t> nact((size_t)H.J, 0), caller_off((size_t)H.J + 1, 0);
        for (int32_t j = 0; j < H.J; j++) nact[H.caller_inf[j]] = H.inf_seq[j + 1] - H.inf_seq[j];
        for (int32_t j = 0; j < H.J; j++) caller_off[j + 1] = caller_off[j] + nact[j];
        for (int32_t j = 0; j < H.J; j++) {
            double sum = 0.0;
            for (int32_t a = caller_off[j]; a < caller_off[j + 1]; a++) {
                if (!(b[a] >= 0.0)) return nfail(CFR_ERR_ARG, "strategy entries must be >= 0");
                sum += b[a];
            }
            if (std::fabs(sum - 1.0) > 1e-5) return nfail(CFR_ERR_ARG, "strategy of an infoset does not sum to 1");
        }
    }
    if (r) {
        std::vector<float2> h(S1, make_float2(0.f, 0.f));
        for (int64_t k = 1; k <= P.S; k++) h[H.seq_of_caller[k]] = ff(r[k - 1]);
        NCU(cudaMemcpy(P.r, h.data(), S1 * sizeof(float2), cudaMemcpyHostToDevice));
    }
    if (xbar) {
        std::vector<float2> h(S1);
        h[0] = ff(xbar[0]);
        for (int64_t k = 1; k <= P.S; k++) h[H.seq_of_caller[k]] = ff(xbar[k]);
        NCU(cudaMemcpy(P.xbar, h.data(), S1 * sizeof(float2), cudaMemcpyHostToDevice));
    }
    if (b) {
        std::vector<float> h(S1, 0.f);
        for (int64_t k = 1; k <= P.S; k++) h[H.seq_of_caller[k]] = (float)b[k - 1];
        NCU(cudaMemcpy(P.b, h.data(), S1 * sizeof(float), cudaMemcpyHostToDevice));
        down(ctx, player);   // the sequence form of the strategy to be played next
    }
    if (t >= 0) {
        const int32_t tt = (int32_t)t;
        NCU(cudaMemcpy(ctx->t_dev, &tt, sizeof(tt), cudaMemcpyHostToDevice));
        ctx->t = t;
    }
    return cfrn_sync(ctx);
}

int cfrn_get_values(cfrn_ctx *ctx, int player, double *x, double *u) {
    if (int rc = check_player(ctx, player)) return rc;
    const NDev &P = ctx->P[player];
    const NPlayerHost &H = ctx->host.pl[player];
    const int64_t S1 = (int64_t)P.S + 1;
    auto fl = [](float v) { return (double)v; };
    if (u) {
        if (int rc = rows(ctx, player, P.uq)) return rc;
    }
    if (int rc = cfrn_sync(ctx)) return rc;
    std::vector<float> h(S1);
    if (x) {
        NCU(cudaMemcpy(h.data(), P.x, S1 * sizeof(float), cudaMemcpyDeviceToHost));
        to_caller(H, h, x, true, fl);
    }
    if (u) {
        NCU(cudaMemcpy(h.data(), P.uq, S1 * sizeof(float), cudaMemcpyDeviceToHost));
        to_caller(H, h, u, true, fl);
    }
    return CFR_OK;
}

int cfrn_get_average_strategy(cfrn_ctx *ctx, int player, double *out, int64_t len) {
    if (int rc = check_player(ctx, player)) return rc;
    const NPlayerHost &H = ctx->host.pl[player];
    if (!out || len != H.S) return nfail(CFR_ERR_ARG, "output length must be S_p");
    std::vector<double> xb((size_t)H.S + 1);
    if (int rc = cfrn_get_state(ctx, player, nullptr, nullptr, xb.data(), nullptr)) return rc;
    // xbar in the caller numbering: decision point j's parent sequence in
    // that numbering is read through the layout's maps
    std::vector<int32_t> caller_of_seq((size_t)H.S + 1, 0);
    for (int32_t k = 1; k <= H.S; k++) caller_of_seq[H.seq_of_caller[k]] = k;
    for (int32_t j = 0; j < H.J; j++) {
        const int32_t s0 = H.inf_seq[j], s1 = H.inf_seq[j + 1];
        const double d = xb[caller_of_seq[H.inf_par[j]]];
        for (int32_t s = s0; s < s1; s++) {
            const int32_t k = caller_of_seq[s];
            out[k - 1] = d > 0.0 ? xb[k] / d : 1.0 / (double)(s1 - s0);
        }
    }
    return CFR_OK;
}

int cfrn_nash_conv(cfrn_ctx *ctx, double *nash_conv, double *gains) {
    if (!ctx || !nash_conv) return nfail(CFR_ERR_ARG, "NULL argument");
    for (int p = 0; p < ctx->n; p++) {
        NDev &P = ctx->P[p];
        k_np_avgnorm<<<blocks(P.S + 1), kThreadsN, 0, ctx->stream>>>(P.xbar, P.x, P.x64, P.S + 1);
        counted(ctx);
    }
    for (int i = 0; i < ctx->n; i++) {
        NDev &P = ctx->P[i];
        if (int rc = rows64(ctx, i)) return rc;
        for (int l = P.L - 1; l >= 0; l--) {
            const int j0 = P.lvl[l], j1 = P.lvl[l + 1];
            k_np_br<<<blocks(j1 - j0), kThreadsN, 0, ctx->stream>>>(P.dp, j0, j1);
            counted(ctx);
        }
        k_np_value<<<1, kThreadsN, 0, ctx->stream>>>(P.x64, P.u64, P.S + 1, P.seq_child, P.ev64, ctx->out + 2 * i);
        counted(ctx);
    }
    NCU(cudaGetLastError());
    double h[2 * kMaxP];
    NCU(cudaMemcpyAsync(h, ctx->out, sizeof(double) * 2 * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    NCU(cudaStreamSynchronize(ctx->stream));
    double sum = 0.0;
    for (int i = 0; i < ctx->n; i++) {
        const double g = h[2 * i + 1] - h[2 * i];
        if (gains) gains[i] = g;
        sum += g;
    }
    *nash_conv = sum;
    return CFR_OK;
}

int cfrn_time_passes(cfrn_ctx *ctx, int iters, int variant, double alpha, double beta, double gamma, int alternating,
                     double *us) {
    if (!ctx || !us) return nfail(CFR_ERR_ARG, "NULL argument");
    if (iters < 1 || variant < 0 || variant > 4) return nfail(CFR_ERR_ARG, "bad iteration count or variant");
    cudaEvent_t ev[4][2 * kMaxP];
    for (auto &row : ev)
        for (auto &e : row) NCU(cudaEventCreate(&e));
    double acc[4] = {0, 0, 0, 0};
    int rc = CFR_OK;
    for (int it = 0; it < iters && rc == CFR_OK; it++) {
        params(ctx, 1, variant, alpha, beta, gamma);
        rc = iteration(ctx, 0, variant, alternating != 0, ev);
        tick(ctx, 1);
        ctx->t += 1;
        if (rc == CFR_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = nfail(CFR_ERR_CUDA, "timing run");
        for (int k = 0; k < 4 && rc == CFR_OK; k++)
            for (int i = 0; i < ctx->n; i++) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[k][2 * i], ev[k][2 * i + 1]);
                acc[k] += ms;
            }
    }
    for (auto &row : ev)
        for (auto &e : row) cudaEventDestroy(e);
    if (rc) return rc;
    for (int k = 0; k < 4; k++) us[k] = acc[k] * 1e3 / iters;
    return CFR_OK;
}

int64_t cfrn_launches(const cfrn_ctx *ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
