// Device building blocks of one sequence-form CFR iteration (sm_103a).
//
// One player's half-step is two persistent launches over the forest layout
// (layout.h), each taking units of work from a queue:
//
//   up   : per unit (a range of subtrees, a few levels deep), deepest level
//          first:
//            - payoff product rows u = sign * M x_other          (Sec. 2.1, two-player utilities)
//            - V[s] = u[s] + sum of the child infosets' ev       (Alg. 2: v += L w + L v; q = B^T(w+v))
//            - ev_j = sum_a b_j[a] V[(j,a)]                       (C (b . q))
//            - r += V - ev_j, variant post-op, next strategy     (Alg. 2 regret update; Alg. 3-5)
//          The queue holds every leaf unit, then the internal units deepest
//          first; an internal unit waits (bounded) until its children have
//          counted themselves done, then copies in their top-level ev.  Once a
//          CTA finds the queue empty it joins the average update
//          xbar += t^gamma x for the strategy x about to be replaced.
//   down : per unit, top-down: x[(j,a)] = x[p_j] b_j[a]          (Alg. 2: y += L^T y; x = A^T y)
//          Each unit first recomputes the next x of its ancestor chain (the
//          infosets above its top level, up to the game's root) from the
//          final b, so the units are independent of one another.
//
// Completion is counted with one atomic per unit (threadfence-reduction
// pattern).  Cumulative regrets and average sums are float-float pairs
// (Kahan-compensated FP32): B300's FP64 rate is far below its FP32 rate, so
// the hot path does no FP64 arithmetic.  The best-response pass (MODE_BR)
// runs in FP64.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "layout.h"

namespace cfrb {

constexpr int kThreads = 256;      // threads of a global-path CTA
constexpr int kStage = 8;          // products staged per lane per pass of the payoff SpMV

enum { VAR_CFR = 0, VAR_PLUS = 1, VAR_DCFR = 2, VAR_PCFR_PLUS = 3, VAR_PCFR = 4 };
// predictive variants: the next strategy is regret matching of r + the
// instantaneous regret just observed (Alg. 5 with m^(t+1) = u^t)
__host__ __device__ constexpr bool predictive(int v) { return v == VAR_PCFR_PLUS || v == VAR_PCFR; }
// MODE_CFR: the FP32 iteration (units too large to stage); MODE_BR: the FP64
// best response; MODE_CFR64: the iteration in FP64 throughout (precision 64)
enum { MODE_CFR = 0, MODE_BR = 1, MODE_CFR64 = 2 };

struct DevPlayer {
    // structure (read-only)
    const int32_t *inf_seq, *seq_child, *inf_par, *seq_game;
    const int32_t *m_ptr, *m_col;
    const float *m_val;
    const double *m_val64;
    const int4 *units;              // {game, nlvl, rng, flags}; ranges: kLvl ints per level
    const int2 *unit_tree;          // {parent unit (-1: root), child units}
    // the queues in order, two int4 per entry: the unit's header
    // {game, nlvl, rng, flags} and {unit, parent, child units, 0}, so a pass
    // reads an entry with two independent loads
    const int4 *upq, *downq;
    const int32_t *ranges, *game_root;
    // the other player's x for a staged level: per-entry gathers, or copied
    // windows of it (rwin: {w0, w1, x-area bytes, 0} per range record; win:
    // {c0, c1, byte offset, level} per window; lcol: the staged columns,
    // local to the level's x area where it has windows)
    const int32_t *lcol;
    const int4 *rwin, *win;
    int32_t n_units, n_up, G;       // n_units: top-down units; n_up: bottom-up queue length
    int32_t S;                      // sequences
    // state
    float2 *r;       // cumulative regret, float-float (hi, lo)
    float *b;        // behavioural strategy to be played next
    float *x;        // sequence-form strategy of the last NextStrategy
    float2 *xbar;    // weighted sum of played x, float-float
    // scratch
    float *xanc;     // top-down units worked from global memory: their ancestors' x
    float *u, *ev;
    double *u64, *ev64, *xnorm;
    // unit_cnt: children completed in the current bottom-up pass (reset by
    // the parent once it has seen them all); qup / qdn: the bottom-up and
    // top-down passes' queue words {head, exit count, launches} (reset by the
    // last CTA to exit a launch; separate words let one pass start while the
    // previous one finishes); err: nonzero once a bounded wait gave up
    int32_t *unit_cnt, *qup, *qdn, *err;
    // qavg: the average pass's chunk queue words {head, exit count, launches}
    int32_t *qavg;
    // root_done[g]: set by the bottom-up loop of a fused half-step once game
    // g's root unit has written b (the launch's top-down epoch + 1)
    int32_t *root_done;
    uint64_t wait_ns;               // longest wait of a unit for the units it depends on
    // precision 64: the state in FP64 (the FP32 state above is then unused)
    int fp64;
    double *r64, *b64, *x64, *xbar64;
    double *evc64;   // ev of every infoset from the last FP64 bottom-up pass
    double *xanc64;  // top-down units: their ancestors' x
};

struct ItemParams;
struct ItemParams64;
struct DevGames {
    int32_t *t_done;        // completed iterations per game
    const uint8_t *active;  // 1 = advance this game
    double *br;             // best-response value per game (BR pass output)
    ItemParams *par;        // [G][kParamSpan + 1] parameters of t = pbase[g] + k
    int32_t *pbase;         // [G]
    int32_t *mixed;         // 0: every game has game 0's parameters in every slot of the table
    ItemParams64 *par64;    // the same table in FP64 (precision 64)
};
constexpr int kParamSpan = 64;   // iterations covered by one parameter table

struct IterArgs {
    int variant;
    int first_of_iter;      // 1 for the first launch of an iteration (player 1's up pass)
    float sign;             // +1: u1 = M y ; -1: u2 = -M^T x
    double alpha, beta, gamma;
    int average;            // down pass: accumulate xbar (0 when only rebuilding x)
    int pslot;              // parameter-table entry of this pass: iteration t = t_done + pslot
                            // at the time the table was filled
    int keep_values;        // up pass: store the ev of every infoset (not only each unit's top level)
};

// ---------------------------------------------------------------------------
// float-float arithmetic (error-free transforms: Knuth two-sum, Dekker)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_add_f(float2 a, float b) {
    float2 s = ff_two_sum(a.x, b);
    return ff_fast_two_sum(s.x, __fadd_rn(s.y, a.y));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float2 s = ff_two_sum(a.x, b.x);
    return ff_fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ float2 ff_mul_f(float2 a, float b) {
    const float p = __fmul_rn(a.x, b);
    const float e = fmaf(a.y, b, fmaf(a.x, b, -p));
    return ff_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ float2 ff_from_double(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// ---------------------------------------------------------------------------
// per-unit parameters (they depend on the game's iteration counter only)
// ---------------------------------------------------------------------------
struct ItemParams {
    float2 w;        // t^gamma
    float2 fpos;     // DCFR: t^alpha / (t^alpha + 1)
    float2 fneg;     // DCFR: t^beta / (t^beta + 1)
    int32_t t;
    int32_t active;
};

// the same in FP64
struct ItemParams64 {
    double w, fpos, fneg;
    int32_t t, active;
};

__device__ __forceinline__ void params_of_t(const DevGames &gm, const IterArgs &ia, int g, int32_t t,
                                            ItemParams *ip, ItemParams64 *ip64 = nullptr) {
    const double td = (double)t;
    ip->t = t;
    ip->active = gm.active[g];
    const double w = pow(td, ia.gamma);
    double fp = 1.0, fn = 1.0;
    ip->w = ff_from_double(w);
    if (ia.variant == VAR_DCFR) {
        const double ta = pow(td, ia.alpha), tb = pow(td, ia.beta);
        fp = ta / (ta + 1.0);
        fn = tb / (tb + 1.0);
        ip->fpos = ff_from_double(fp);
        ip->fneg = ff_from_double(fn);
    } else {
        ip->fpos = make_float2(1.f, 0.f);
        ip->fneg = make_float2(1.f, 0.f);
    }
    if (ip64) *ip64 = ItemParams64{w, fp, fn, t, ip->active};
}
__device__ __forceinline__ void item_params(const DevGames &gm, const IterArgs &ia, int g, ItemParams *ip) {
    params_of_t(gm, ia, g, gm.t_done[g] + (ia.first_of_iter ? 1 : 0), ip);
}
// The parameters of game g for this pass, from the table filled ahead of the
// iterations (FP64 pow is slow on this part and costs registers: the table
// keeps it out of the passes).  The host refills the table every kParamSpan
// iterations and gives each pass its entry, so the lookup depends on no
// counter another kernel writes.
__device__ __forceinline__ ItemParams unit_params(const DevGames &gm, const IterArgs &ia, int g) {
    return gm.par[(int64_t)g * (kParamSpan + 1) + ia.pslot];
}

// ---------------------------------------------------------------------------
// payoff product rows: u[s] = sign * sum_k val[k] * xo[col[k]] for s in the
// sequence ranges of the given unit levels (kLvl ints each).  Each warp owns
// groups of 32 consecutive rows, reads their contiguous nonzeros with
// coalesced loads, stages the products in shared memory and lets each lane
// sum its own row in CSR order (deterministic).
// ---------------------------------------------------------------------------
template <typename T, typename TV>
__device__ void spmv_ranges(const int32_t *__restrict__ m_ptr, const int32_t *__restrict__ m_col,
                            const TV *__restrict__ m_val, const T *__restrict__ xo, T *__restrict__ u,
                            const int32_t *lvls, int n_lvls, T sign, T *stage_all) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    T *stage = stage_all + warp * (32 * kStage);
    int gbase = 0;
    for (int q = 0; q < n_lvls; q++) {
        const int slo = lvls[kLvl * q + 2], shi = lvls[kLvl * q + 3];
        const int ng = (shi - slo + 31) >> 5;
        // group k of this range is handled by warp (gbase + k) % nw
        int k0 = (warp - gbase) % nw;
        if (k0 < 0) k0 += nw;
        for (int k = k0; k < ng; k += nw) {
            const int row = slo + (k << 5) + lane;
            const bool has = row < shi;
            const int p0 = has ? __ldg(&m_ptr[row]) : 0;
            const int p1 = has ? __ldg(&m_ptr[row + 1]) : 0;
            const int last = min(31, shi - 1 - slo - (k << 5));
            const int g0 = __shfl_sync(0xffffffffu, p0, 0);
            const int g1 = __shfl_sync(0xffffffffu, p1, last);
            T acc = T(0);
            for (int base = g0; base < g1; base += 32 * kStage) {
#pragma unroll
                for (int e = 0; e < kStage; e++) {
                    const int kk = base + e * 32 + lane;
                    T prod = T(0);
                    if (kk < g1) prod = T(__ldg(&m_val[kk])) * __ldg(&xo[__ldg(&m_col[kk])]);
                    stage[e * 32 + lane] = prod;
                }
                __syncwarp();
                const int lo = max(p0, base), hi = min(p1, base + 32 * kStage);
                for (int kk = lo; kk < hi; kk++) acc += stage[kk - base];
                __syncwarp();
            }
            if (has) u[row] = sign * acc;
        }
        gbase += ng;
    }
}

// ---------------------------------------------------------------------------
// bottom-up step for one infoset j (MODE_CFR, global memory): counterfactual
// values, regret update, variant post-op and the next behavioural strategy.
// ---------------------------------------------------------------------------
// The variant's post-op on an updated cumulative regret (Alg. 3: floor at 0;
// Alg. 4: discount positive regrets by fpos, negative ones by fneg; Alg. 5:
// floor at 0).  Selects only, so the lanes of a warp never split on the sign
// of r; VAR is a compile-time constant in the staged passes.
template <int VAR>
__device__ __forceinline__ float2 post_op_v(float2 r, float2 fpos, float2 fneg) {
    if (VAR == VAR_PLUS || VAR == VAR_PCFR_PLUS) {
        r = r.x < 0.f ? make_float2(0.f, 0.f) : r;
    } else if (VAR == VAR_DCFR) {
        const float2 f = r.x > 0.f ? fpos : (r.x < 0.f ? fneg : make_float2(1.f, 0.f));
        r = ff_mul(r, f);
    }
    return r;
}
__device__ __forceinline__ float2 post_op(float2 r, int variant, const ItemParams &ip) {
    switch (variant) {
    case VAR_PLUS: return post_op_v<VAR_PLUS>(r, ip.fpos, ip.fneg);
    case VAR_DCFR: return post_op_v<VAR_DCFR>(r, ip.fpos, ip.fneg);
    case VAR_PCFR_PLUS: return post_op_v<VAR_PCFR_PLUS>(r, ip.fpos, ip.fneg);
    default: return r;
    }
}

// Regret matching's normaliser 1/sum(positive regrets): the hardware
// reciprocal (rcp.approx.f32, within 1 ulp, subnormal inputs kept).  Every
// path (staged, wide, global) uses this same instruction, so a sequence's
// strategy does not depend on which path computed it.
__device__ __forceinline__ float rm_inverse(float pos) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(pos));
    return r;
}
// Regrets scale with the opponent's reach, which can fall below FP32's
// normal range deep in a game once the strategies sharpen; the reciprocal of a
// positive sum below 2^-128 would overflow to infinity (and q * inf = NaN for
// the other actions).  So sums below 2^-64 are first scaled by 2^64, exactly,
// and so is each clipped regret q: b = (q sc) / (pos sc) = q / pos, with a
// finite normaliser (pos sc >= 2^-85).  Sums at or above 2^-64 take sc = 1.
struct RmNorm {
    float inv, sc;
};
__device__ __forceinline__ RmNorm rm_norm(float pos) {
    const float sc = pos < 0x1p-64f ? 0x1p64f : 1.f;
    return RmNorm{pos > 0.f ? rm_inverse(pos * sc) : 0.f, sc};
}
__device__ __forceinline__ float rm_prob(float q, const RmNorm &n) { return (q * n.sc) * n.inv; }
// the uniform probability 1/na, correctly rounded (the constants are the
// compiler's correctly rounded quotients)
__device__ __forceinline__ float uniform_prob(int na) {
    return na <= 2 ? (na == 1 ? 1.f : 0.5f) : (na == 3 ? 1.f / 3.f : (na == 4 ? 0.25f : __frcp_rn((float)na)));
}

// V[s] = u[s] + ev of each child infoset, added in child order
__device__ __forceinline__ float value_of(const DevPlayer &P, int s) {
    float v = P.u[s];
    const int c0 = P.seq_child[s], c1 = P.seq_child[s + 1];
    for (int c = c0; c < c1; c++) v += __ldcg(&P.ev[c]);
    return v;
}

__device__ inline void up_infoset_cfr(const DevPlayer &P, int j, int variant, const ItemParams &ip) {
    const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
    const int na = s1 - s0;
    const bool pred = predictive(variant);
    float ev = 0.f;
    for (int s = s0; s < s1; s++) {
        const float v = value_of(P, s);
        P.u[s] = v;   // u is scratch: keep V for the next passes
        ev = fmaf(P.b[s], v, ev);
    }
    P.ev[j] = ev;
    float pos = 0.f;
    for (int s = s0; s < s1; s++) {
        const float d = P.u[s] - ev;
        float2 r = ff_add_f(P.r[s], d);
        r = post_op(r, variant, ip);
        P.r[s] = r;
        const float rr = pred ? r.x + d : r.x;
        const float q = rr > 0.f ? rr : 0.f;
        P.u[s] = q;
        pos += q;
    }
    const RmNorm nrm = rm_norm(pos);
    const float uni = uniform_prob(na);
    for (int s = s0; s < s1; s++) P.b[s] = pos > 0.f ? rm_prob(P.u[s], nrm) : uni;
}

// the bottom-up step in FP64 (precision 64): the same arithmetic as
// up_infoset_cfr on the FP64 state, with regret matching's division exact
// (IEEE) and the FP64 parameters
__device__ inline void up_infoset_cfr64(const DevPlayer &P, int j, int variant, const ItemParams64 &ip) {
    const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
    const bool pred = predictive(variant);
    double ev = 0.0;
    for (int s = s0; s < s1; s++) {
        double v = P.u64[s];
        const int c0 = P.seq_child[s], c1 = P.seq_child[s + 1];
        for (int c = c0; c < c1; c++) v += __ldcg(&P.evc64[c]);
        P.u64[s] = v;   // u is scratch: keep V for the next loops
        ev += P.b64[s] * v;
    }
    P.evc64[j] = ev;
    double pos = 0.0;
    for (int s = s0; s < s1; s++) {
        const double d = P.u64[s] - ev;
        double r = P.r64[s] + d;
        if (variant == VAR_PLUS || variant == VAR_PCFR_PLUS) r = r < 0.0 ? 0.0 : r;
        else if (variant == VAR_DCFR) r = r > 0.0 ? r * ip.fpos : (r < 0.0 ? r * ip.fneg : r);
        P.r64[s] = r;
        const double rr = pred ? r + d : r;
        const double q = rr > 0.0 ? rr : 0.0;
        P.u64[s] = q;
        pos += q;
    }
    const double uni = 1.0 / (double)(s1 - s0);
    for (int s = s0; s < s1; s++) P.b64[s] = pos > 0.0 ? P.u64[s] / pos : uni;
}

// best-response step (MODE_BR, FP64): V = u + sum children, ev = max_a V
__device__ inline void up_infoset_br(const DevPlayer &P, int j) {
    const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
    double best = -INFINITY;
    for (int s = s0; s < s1; s++) {
        double v = P.u64[s];
        const int c0 = P.seq_child[s], c1 = P.seq_child[s + 1];
        for (int c = c0; c < c1; c++) v += __ldcg(&P.ev64[c]);
        best = v > best ? v : best;
    }
    P.ev64[j] = best;
}

// Levels of one unit bottom-up (deepest first), after its payoff rows,
// straight from global memory (units too large to stage, and the
// best-response pass).  rng: kLvl ints per level.
template <int MODE>
__device__ void run_up(const DevPlayer &P, const void *xo, const IterArgs &ia, const ItemParams &ip, int nlvl,
                       const int32_t *rng, void *stage, const ItemParams64 *ip64 = nullptr) {
    if (MODE == MODE_CFR)
        spmv_ranges<float, float>(P.m_ptr, P.m_col, P.m_val, (const float *)xo, P.u, rng, nlvl, ia.sign,
                                  (float *)stage);
    else
        spmv_ranges<double, double>(P.m_ptr, P.m_col, P.m_val64, (const double *)xo, P.u64, rng, nlvl,
                                    (double)ia.sign, (double *)stage);
    __syncthreads();
    for (int k = nlvl - 1; k >= 0; k--) {
        const int jlo = rng[kLvl * k], jhi = rng[kLvl * k + 1];
        for (int j = jlo + (int)threadIdx.x; j < jhi; j += blockDim.x) {
            if (MODE == MODE_CFR) up_infoset_cfr(P, j, ia.variant, ip);
            else if (MODE == MODE_CFR64) up_infoset_cfr64(P, j, ia.variant, *ip64);
            else up_infoset_br(P, j);
        }
        __syncthreads();
    }
}

}  // namespace cfrb
