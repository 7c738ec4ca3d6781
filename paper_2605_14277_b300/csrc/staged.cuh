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

// Thread 0 only: lay out a unit in buffer `buf` and start its copies.  The
// shared tables are filled and the bytes counted first, then the barrier is
// armed and the copies issued.
__device__ void issue_up(const DevPlayer &P, const int4 hdr, unsigned char *buf, uint64_t *bar, SLvl *lv,
                         UpTab *tab) {
    const int32_t *rng = P.ranges + hdr.z;
    const int nl = hdr.y;
    const void *src[kMaxStagedLevels][7];
    uint32_t nb[kMaxStagedLevels][7];
    uint32_t total = 0;
    unsigned char *cur = buf;
    for (int k = 0; k < nl; k++) {
        const int32_t *d = rng + kLvl * k;
        const SLvl L{d[0], d[1], d[2], d[3], d[4], d[5]};
        lv[k] = L;
        UpTab &t = tab[k];
        t.r = (float2 *)place(cur, P.r, L.s0, L.s1, 8, &src[k][0], &nb[k][0]);
        t.b = (float *)place(cur, P.b, L.s0, L.s1, 4, &src[k][1], &nb[k][1]);
        t.sch = (const int32_t *)place(cur, P.seq_child, L.s0, L.s1 + 1, 4, &src[k][2], &nb[k][2]);
        t.mptr = (const int32_t *)place(cur, P.m_ptr, L.s0, L.s1 + 1, 4, &src[k][3], &nb[k][3]);
        t.iseq = (const int32_t *)place(cur, P.inf_seq, L.j0, L.j1 + 1, 4, &src[k][4], &nb[k][4]);
        t.col = (const int32_t *)place(cur, P.m_col, L.n0, L.n1, 4, &src[k][5], &nb[k][5]);
        t.val = (float *)place(cur, P.m_val, L.n0, L.n1, 4, &src[k][6], &nb[k][6]);
        t.V = (float *)cur;
        cur += work16(L.s1 - L.s0, 4);
        t.ev = (float *)cur;
        cur += work16(L.j1 - L.j0, 4);
        for (int f = 0; f < 7; f++) total += nb[k][f];
    }
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, total);
    for (int k = 0; k < nl; k++) {
        const void *dsts[7] = {tab[k].r, tab[k].b, tab[k].sch, tab[k].mptr, tab[k].iseq, tab[k].col, tab[k].val};
        for (int f = 0; f < 7; f++)
            if (nb[k][f]) {
                // the reserved span starts 16-aligned; the element pointer sits
                // at the same offset from it as the source element from A
                void *d0 = (void *)(((uintptr_t)dsts[f]) & ~(uintptr_t)15);
                bulk_g2s(d0, src[k][f], nb[k][f], bar);
            }
    }
}

__device__ void issue_down(const DevPlayer &P, const int4 hdr, unsigned char *buf, uint64_t *bar, SLvl *lv,
                           DownTab *tab) {
    const int32_t *rng = P.ranges + hdr.z;
    const int nl = hdr.y;
    const void *src[kMaxStagedLevels][5];
    uint32_t nb[kMaxStagedLevels][5];
    uint32_t total = 0;
    unsigned char *cur = buf;
    for (int k = 0; k < nl; k++) {
        const int32_t *d = rng + kLvl * k;
        const SLvl L{d[0], d[1], d[2], d[3], d[4], d[5]};
        lv[k] = L;
        DownTab &t = tab[k];
        t.b = (float *)place(cur, P.b, L.s0, L.s1, 4, &src[k][0], &nb[k][0]);
        t.x = (float *)place(cur, P.x, L.s0, L.s1, 4, &src[k][1], &nb[k][1]);
        t.xbar = (float2 *)place(cur, P.xbar, L.s0, L.s1, 8, &src[k][2], &nb[k][2]);
        t.ipar = (const int32_t *)place(cur, P.inf_par, L.j0, L.j1, 4, &src[k][3], &nb[k][3]);
        t.iseq = (const int32_t *)place(cur, P.inf_seq, L.j0, L.j1 + 1, 4, &src[k][4], &nb[k][4]);
        for (int f = 0; f < 5; f++) total += nb[k][f];
    }
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, total);
    for (int k = 0; k < nl; k++) {
        const void *dsts[5] = {tab[k].b, tab[k].x, tab[k].xbar, tab[k].ipar, tab[k].iseq};
        for (int f = 0; f < 5; f++)
            if (nb[k][f]) {
                void *d0 = (void *)(((uintptr_t)dsts[f]) & ~(uintptr_t)15);
                bulk_g2s(d0, src[k][f], nb[k][f], bar);
            }
    }
}

// Up pass of a staged unit: payoff rows, bottom-up values, regret update,
// variant post-op and next strategy, all in shared memory; then write-back.
__device__ void compute_up(const DevPlayer &P, const float *__restrict__ xo, const IterArgs &ia,
                           const ItemParams &ip, int nl, const SLvl *lv, const UpTab *tab) {
    const int tid = threadIdx.x, nt = blockDim.x;
    // products val * xo[col], in place (gathers of the other player's x)
    for (int k = 0; k < nl; k++) {
        const int nz = lv[k].n1 - lv[k].n0;
        float *val = tab[k].val;
        const int32_t *col = tab[k].col;
        for (int q = tid; q < nz; q += nt) val[q] *= __ldg(&xo[col[q]]);
    }
    __syncthreads();
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
    __syncthreads();
    const bool pred = (ia.variant == VAR_PCFR_PLUS);
    for (int k = nl - 1; k >= 0; k--) {
        const SLvl L = lv[k];
        const UpTab t = tab[k];
        const int ni = L.j1 - L.j0;
        const int cj0 = (k + 1 < nl) ? lv[k + 1].j0 : 0;
        const float *evc = (k + 1 < nl) ? tab[k + 1].ev : nullptr;
        for (int i = tid; i < ni; i += nt) {
            const int q0 = t.iseq[i] - L.s0, q1 = t.iseq[i + 1] - L.s0;
            float ev = 0.f;
            for (int q = q0; q < q1; q++) {
                float v = t.V[q];
                for (int c = t.sch[q] - cj0; c < t.sch[q + 1] - cj0; c++) v += evc[c];
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
        __syncthreads();
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
    const int tid = threadIdx.x, nt = blockDim.x;
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
        __syncthreads();
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
