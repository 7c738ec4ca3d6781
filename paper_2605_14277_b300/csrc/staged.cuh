// Shared-memory staged work units for the two per-player passes.
//
// A work unit (layout.h) is one contiguous range per level of every array it
// touches, so one thread can copy the whole unit into shared memory with bulk
// asynchronous copies (cp.async.bulk, completion counted in bytes on an
// mbarrier) before any index is read.  The CTA then runs the unit's levels
// out of shared memory and writes its results back with coalesced stores.
// Two buffers per CTA: the next unit's copies are in flight while the current
// one is computed.
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace cfrb {

constexpr int kThreadsS = 512;              // threads of a staged CTA (one CTA per SM)
constexpr uint32_t kWaitLimit = 1u << 26;   // polls of an mbarrier before giving up
constexpr int kErrTimeout = 1;

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false (and the error word set) if the phase never completes
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int32_t *err) {
    for (uint32_t k = 0; k < kWaitLimit; k++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (k > 64) __nanosleep(64);
    }
    atomicExch(err, kErrTimeout);
    return false;
}

// Warp 0 of a staged CTA is the producer (queue fetches, bulk-copy issue);
// warps 1.. compute, synchronising among themselves on named barrier 1.
constexpr int kProducerThreads = 32;
__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"r"((int)blockDim.x - kProducerThreads) : "memory");
}

// Per-iteration parameters depend on the game only through its iteration
// counter t, so a CTA keeps the last set it computed (FP64 pow on B300 is slow).
struct ParamCache {
    int32_t t;
    ItemParams p;
};
__device__ __forceinline__ void cached_params(const DevGames &gm, const IterArgs &ia, int g, ParamCache *c,
                                              ItemParams *out) {
    const int32_t t = gm.t_done[g] + (ia.first_of_iter ? 1 : 0);
    if (t != c->t) {
        item_params(gm, ia, g, &c->p);
        c->t = t;
    }
    *out = c->p;
    out->t = t;
    out->active = gm.active[g];
}

// one unit level as staged in shared memory
struct SLvl {
    int32_t j0, j1, s0, s1, n0, n1;
};

// shared-memory pointers of one staged level
struct UpTab {
    float2 *r;
    float *b;
    const int32_t *sch, *mptr, *iseq, *col;
    float *val;     // payoff values, overwritten in place by the products
    float *V;       // u, then counterfactual values, then clipped regrets
    float *ev;
};
struct DownTab {
    float *b, *x;
    float2 *xbar;
    const int32_t *ipar, *iseq;
};

// reserve the copied range [a, b) of an array with element size e at gbase;
// returns the shared pointer of element a and, in *src/*bytes, the aligned copy
__device__ __forceinline__ unsigned char *place(unsigned char *&cur, const void *gbase, int64_t a, int64_t b, int e,
                                                const void **src, uint32_t *bytes) {
    const uintptr_t g0 = (uintptr_t)gbase + (uintptr_t)(a * e);
    const uintptr_t g1 = (uintptr_t)gbase + (uintptr_t)(b * e);
    const uintptr_t A = g0 & ~(uintptr_t)15;
    const uintptr_t B = (g1 + 15) & ~(uintptr_t)15;
    unsigned char *dst = cur;
    cur += span16(b - a, e);
    *src = (const void *)A;
    *bytes = (b > a) ? (uint32_t)(B - A) : 0u;
    return dst + (g0 - A);
}

// Warp 0 (all 32 lanes): lay out a unit in buffer `buf` and start its copies.
// Lane k owns level k: it sizes the level (the same formula the host packer
// used), a warp scan places the levels one after another, lane 0 arms the
// barrier with the total byte count, then every lane issues its level's copies.
__device__ void issue_up(const DevPlayer &P, const int4 hdr, unsigned char *buf, uint64_t *bar, SLvl *lv,
                         UpTab *tab) {
    const int lane = threadIdx.x & 31;
    const int32_t *rng = P.ranges + hdr.z;
    const int nl = hdr.y;
    SLvl L{0, 0, 0, 0, 0, 0};
    int64_t bytes = 0;
    if (lane < nl) {
        const int32_t *d = rng + kLvl * lane;
        L = SLvl{d[0], d[1], d[2], d[3], d[4], d[5]};
        bytes = up_level_bytes(L.s1 - L.s0, L.j1 - L.j0, L.n1 - L.n0);
    }
    int64_t off = bytes;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
    }
    off -= bytes;   // exclusive prefix: this level's start
    const void *src[7];
    uint32_t nb[7] = {0, 0, 0, 0, 0, 0, 0};
    uint32_t mine = 0;
    if (lane < nl) {
        unsigned char *cur = buf + off;
        lv[lane] = L;
        UpTab t;
        t.r = (float2 *)place(cur, P.r, L.s0, L.s1, 8, &src[0], &nb[0]);
        t.b = (float *)place(cur, P.b, L.s0, L.s1, 4, &src[1], &nb[1]);
        t.sch = (const int32_t *)place(cur, P.seq_child, L.s0, L.s1 + 1, 4, &src[2], &nb[2]);
        t.mptr = (const int32_t *)place(cur, P.m_ptr, L.s0, L.s1 + 1, 4, &src[3], &nb[3]);
        t.iseq = (const int32_t *)place(cur, P.inf_seq, L.j0, L.j1 + 1, 4, &src[4], &nb[4]);
        t.col = (const int32_t *)place(cur, P.m_col, L.n0, L.n1, 4, &src[5], &nb[5]);
        t.val = (float *)place(cur, P.m_val, L.n0, L.n1, 4, &src[6], &nb[6]);
        t.V = (float *)cur;
        cur += work16(L.s1 - L.s0, 4);
        t.ev = (float *)cur;
        tab[lane] = t;
        for (int f = 0; f < 7; f++) mine += nb[f];
    }
    uint32_t total = mine;
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    fence_proxy_async();
    if (lane == 0) mbar_arrive_expect_tx(bar, total);
    __syncwarp();
    if (lane < nl) {
        const UpTab &t = tab[lane];
        const void *dsts[7] = {t.r, t.b, t.sch, t.mptr, t.iseq, t.col, t.val};
        for (int f = 0; f < 7; f++)
            if (nb[f]) bulk_g2s((void *)(((uintptr_t)dsts[f]) & ~(uintptr_t)15), src[f], nb[f], bar);
    }
}

__device__ void issue_down(const DevPlayer &P, const int4 hdr, unsigned char *buf, uint64_t *bar, SLvl *lv,
                           DownTab *tab) {
    const int lane = threadIdx.x & 31;
    const int32_t *rng = P.ranges + hdr.z;
    const int nl = hdr.y;
    SLvl L{0, 0, 0, 0, 0, 0};
    int64_t bytes = 0;
    if (lane < nl) {
        const int32_t *d = rng + kLvl * lane;
        L = SLvl{d[0], d[1], d[2], d[3], d[4], d[5]};
        bytes = down_level_bytes(L.s1 - L.s0, L.j1 - L.j0);
    }
    int64_t off = bytes;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
    }
    off -= bytes;
    const void *src[5];
    uint32_t nb[5] = {0, 0, 0, 0, 0};
    uint32_t mine = 0;
    if (lane < nl) {
        unsigned char *cur = buf + off;
        lv[lane] = L;
        DownTab t;
        t.b = (float *)place(cur, P.b, L.s0, L.s1, 4, &src[0], &nb[0]);
        t.x = (float *)place(cur, P.x, L.s0, L.s1, 4, &src[1], &nb[1]);
        t.xbar = (float2 *)place(cur, P.xbar, L.s0, L.s1, 8, &src[2], &nb[2]);
        t.ipar = (const int32_t *)place(cur, P.inf_par, L.j0, L.j1, 4, &src[3], &nb[3]);
        t.iseq = (const int32_t *)place(cur, P.inf_seq, L.j0, L.j1 + 1, 4, &src[4], &nb[4]);
        tab[lane] = t;
        for (int f = 0; f < 5; f++) mine += nb[f];
    }
    uint32_t total = mine;
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    fence_proxy_async();
    if (lane == 0) mbar_arrive_expect_tx(bar, total);
    __syncwarp();
    if (lane < nl) {
        const DownTab &t = tab[lane];
        const void *dsts[5] = {t.b, t.x, t.xbar, t.ipar, t.iseq};
        for (int f = 0; f < 5; f++)
            if (nb[f]) bulk_g2s((void *)(((uintptr_t)dsts[f]) & ~(uintptr_t)15), src[f], nb[f], bar);
    }
}

// Up pass of a staged unit (consumer warps only): payoff rows, bottom-up
// values, regret update, variant post-op and next strategy, all in shared
// memory; then write-back.  For a trunk, the deepest level's children are the
// work items' top-level infosets, read from global memory.
constexpr int kRegA = 4;   // infosets with at most kRegA actions keep their values in registers

__device__ __forceinline__ void up_step_reg(const UpTab &t, const SLvl &L, int i, int q0, int na, int cj0,
                                            const float *evc, bool glob, int variant, bool pred,
                                            const ItemParams &ip) {
    float V[kRegA], bb[kRegA], qv[kRegA];
    int cc[kRegA + 1];
    float2 rr[kRegA];
#pragma unroll
    for (int a = 0; a < kRegA; a++)
        if (a < na) {
            V[a] = t.V[q0 + a];
            bb[a] = t.b[q0 + a];
            rr[a] = t.r[q0 + a];
        }
#pragma unroll
    for (int a = 0; a <= kRegA; a++)
        if (a <= na) cc[a] = t.sch[q0 + a] - cj0;
#pragma unroll
    for (int a = 0; a < kRegA; a++)
        if (a < na)
            for (int c = cc[a]; c < cc[a + 1]; c++) V[a] += glob ? __ldcg(&evc[c]) : evc[c];
    float ev = 0.f;
#pragma unroll
    for (int a = 0; a < kRegA; a++)
        if (a < na) ev = fmaf(bb[a], V[a], ev);
    t.ev[i] = ev;
    float pos = 0.f;
#pragma unroll
    for (int a = 0; a < kRegA; a++)
        if (a < na) {
            const float d = V[a] - ev;
            float2 r = ff_add_f(rr[a], d);
            r = post_op(r, variant, ip);
            t.r[q0 + a] = r;
            const float x = pred ? r.x + d : r.x;
            qv[a] = x > 0.f ? x : 0.f;
            pos += qv[a];
        }
    const float inv = pos > 0.f ? 1.0f / pos : 0.f;
    const float uni = 1.0f / (float)na;
#pragma unroll
    for (int a = 0; a < kRegA; a++)
        if (a < na) t.b[q0 + a] = pos > 0.f ? qv[a] * inv : uni;
}

__device__ void compute_up(const DevPlayer &P, const float *__restrict__ xo, const IterArgs &ia,
                           const ItemParams &ip, int nl, const SLvl *lv, const UpTab *tab, bool trunk) {
    const int tid = threadIdx.x - kProducerThreads, nt = blockDim.x - kProducerThreads;
    // products val * xo[col], in place (gathers of the other player's x),
    // four independent gathers in flight per thread
    for (int k = 0; k < nl; k++) {
        const int nz = lv[k].n1 - lv[k].n0;
        float *val = tab[k].val;
        const int32_t *col = tab[k].col;
        for (int q = tid; q < nz; q += 4 * nt) {
            float g[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int e = q + u * nt;
                g[u] = e < nz ? __ldg(&xo[col[e]]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int e = q + u * nt;
                if (e < nz) val[e] *= g[u];
            }
        }
    }
    consumer_sync();
    // row sums in CSR order
    for (int k = 0; k < nl; k++) {
        const int ns = lv[k].s1 - lv[k].s0, n0 = lv[k].n0;
        const float *val = tab[k].val;
        const int32_t *mp = tab[k].mptr;
        float *V = tab[k].V;
        for (int q = tid; q < ns; q += nt) {
            float acc = 0.f;
            for (int e = mp[q] - n0; e < mp[q + 1] - n0; e++) acc += val[e];
            V[q] = ia.sign * acc;
        }
    }
    consumer_sync();
    const bool pred = (ia.variant == VAR_PCFR_PLUS);
    for (int k = nl - 1; k >= 0; k--) {
        const SLvl L = lv[k];
        const UpTab t = tab[k];
        const int ni = L.j1 - L.j0;
        // children of this level: the unit's next level in shared memory, or
        // (a trunk's deepest level) the work items' top levels in global memory
        const bool glob = (k + 1 == nl) && trunk;
        const int cj0 = glob ? 0 : ((k + 1 < nl) ? lv[k + 1].j0 : 0);
        const float *evc = glob ? P.ev : ((k + 1 < nl) ? tab[k + 1].ev : nullptr);
        for (int i = tid; i < ni; i += nt) {
            const int q0 = t.iseq[i] - L.s0, q1 = t.iseq[i + 1] - L.s0;
            if (q1 - q0 <= kRegA) {
                up_step_reg(t, L, i, q0, q1 - q0, cj0, evc, glob, ia.variant, pred, ip);
                continue;
            }
            float ev = 0.f;
            for (int q = q0; q < q1; q++) {
                float v = t.V[q];
                for (int c = t.sch[q] - cj0; c < t.sch[q + 1] - cj0; c++) v += glob ? __ldcg(&evc[c]) : evc[c];
                t.V[q] = v;
                ev = fmaf(t.b[q], v, ev);
            }
            t.ev[i] = ev;
            float pos = 0.f;
            for (int q = q0; q < q1; q++) {
                const float d = t.V[q] - ev;
                float2 r = ff_add_f(t.r[q], d);
                r = post_op(r, ia.variant, ip);
                t.r[q] = r;
                const float rr = pred ? r.x + d : r.x;
                const float qq = rr > 0.f ? rr : 0.f;
                t.V[q] = qq;   // V is no longer needed: keep the clipped regret
                pos += qq;
            }
            const float inv = pos > 0.f ? 1.0f / pos : 0.f;
            const float uni = 1.0f / (float)(q1 - q0);
            for (int q = q0; q < q1; q++) t.b[q] = pos > 0.f ? t.V[q] * inv : uni;
        }
        consumer_sync();
    }
    // write-back (coalesced)
    for (int k = 0; k < nl; k++) {
        const SLvl L = lv[k];
        const int ns = L.s1 - L.s0;
        for (int q = tid; q < ns; q += nt) {
            P.r[L.s0 + q] = tab[k].r[q];
            P.b[L.s0 + q] = tab[k].b[q];
        }
    }
    if (nl > 0) {
        const int ni = lv[0].j1 - lv[0].j0;
        for (int i = tid; i < ni; i += nt) P.ev[lv[0].j0 + i] = tab[0].ev[i];
    }
}

// Down pass of a staged unit: x[(j,a)] = x[p_j] b_j[a] top-down (the top
// level's parents are trunk sequences, read from the staging vector xn), and
// xbar += w x for the strategy being replaced.
__device__ void compute_down(const DevPlayer &P, const IterArgs &ia, const ItemParams &ip, int nl, const SLvl *lv,
                             const DownTab *tab) {
    const int tid = threadIdx.x - kProducerThreads, nt = blockDim.x - kProducerThreads;
    const bool avg = ia.average != 0;
    for (int k = 0; k < nl; k++) {
        const SLvl L = lv[k];
        const DownTab t = tab[k];
        const int ni = L.j1 - L.j0;
        const int ps0 = (k > 0) ? lv[k - 1].s0 : 0;
        const float *xpar = (k > 0) ? tab[k - 1].x : nullptr;
        for (int i = tid; i < ni; i += nt) {
            const int par = t.ipar[i];
            const float xp = (k == 0) ? __ldcg(&P.xn[par]) : xpar[par - ps0];
            for (int q = t.iseq[i] - L.s0; q < t.iseq[i + 1] - L.s0; q++) {
                if (avg) t.xbar[q] = ff_add(t.xbar[q], ff_mul_f(ip.w, t.x[q]));
                t.x[q] = xp * t.b[q];
            }
        }
        consumer_sync();
    }
    for (int k = 0; k < nl; k++) {
        const SLvl L = lv[k];
        const int ns = L.s1 - L.s0;
        for (int q = tid; q < ns; q += nt) {
            P.x[L.s0 + q] = tab[k].x[q];
            if (avg) P.xbar[L.s0 + q] = tab[k].xbar[q];
        }
    }
}

}  // namespace cfrb
