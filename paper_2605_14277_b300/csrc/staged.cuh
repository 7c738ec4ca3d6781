// Shared-memory staged units for the two per-player passes.
//
// A unit (layout.h) is one contiguous range per level of every array it
// touches, so the producer warp can copy the whole unit into shared memory
// with bulk asynchronous copies (cp.async.bulk, completion counted in bytes on
// an mbarrier) before any index is read.  The consumer warps then run the
// unit's levels out of shared memory and write the results back with
// coalesced stores.  Two buffers per CTA: the next unit's copies are in
// flight while the current one is computed, and several CTAs share an SM.
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace cfrb {

constexpr uint32_t kWaitLimit = 1u << 26;          // polls of an mbarrier before giving up
constexpr uint64_t kFlagWaitNs = 1000000000ull;    // longest wait for a parent unit (1 s)
constexpr int kErrTimeout = 1;
constexpr uint32_t kChunk = 4096;                  // bulk copies above this size are split across the warp

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// order this thread's (and, through a preceding barrier or acquire, other
// threads') generic-proxy accesses before its later bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
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
// 4-byte asynchronous global -> shared copy (one gathered element)
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int32_t *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// bounded wait for *flag == want (one thread): false (and the error word set)
// if it does not happen within kFlagWaitNs
__device__ __forceinline__ bool flag_wait(const int32_t *flag, int want, int32_t *err) {
    if (ld_acquire(flag) == want) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t k = 0;; k++) {
        __nanosleep(k < 16 ? 32 : 256);
        if (ld_acquire(flag) == want) return true;
        if ((k & 63) == 63 && globaltimer() - t0 > kFlagWaitNs) break;
    }
    atomicExch(err, kErrTimeout);
    return false;
}

// Warp 0 of a staged CTA is the producer (queue fetches, bulk-copy issue,
// parameter loads); warps 1.. compute, synchronising among themselves on
// named barrier 1.
constexpr int kProducerThreads = 32;
__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"r"((int)blockDim.x - kProducerThreads) : "memory");
}

// one unit level as staged in shared memory
struct SLvl {
    int32_t j0, j1, s0, s1, n0, n1;
};

// The arrays of one staged level, as byte offsets into the CTA's dynamic
// shared memory: 32-bit shared addresses keep the loads on the shared-memory
// path (no generic-address conversion) and halve the registers they take.
template <class T>
__device__ __forceinline__ T *sh(uint32_t off) {
    extern __shared__ __align__(128) unsigned char smem[];
    return reinterpret_cast<T *>(smem + off);
}
__device__ __forceinline__ uint32_t sh_off(const void *p) {
    extern __shared__ __align__(128) unsigned char smem[];
    return (uint32_t)((const unsigned char *)p - smem);
}
struct UpTab {
    uint32_t r;     // float2 cumulative regrets
    uint32_t b;     // float strategy
    uint32_t sch, mptr, iseq, col;   // int32 index arrays
    uint32_t val;   // float payoff values
    uint32_t gx;    // float x of the other player at each payoff entry's column (gathered)
    uint32_t V;     // float counterfactual values, then clipped regrets, then (root) next x
    uint32_t ev;    // float ev per infoset
};
struct DownTab {
    uint32_t b, x;  // float
    uint32_t xbar;  // float2
    uint32_t ipar, iseq;
};
// an internal unit's staged child values: ev of infosets [c0, c1), brought in
// by one bulk copy (dst, src, bytes) once all its children are done
struct ChildEv {
    uint32_t ev;
    int32_t c0;
    uint32_t dst, bytes;
    const void *src;
};

// Shared-memory placement of the copied range [a, b) of an array with element
// size e at gbase: the shared pointer of element a, and the 16-byte aligned
// copy (*dst, *src, *bytes) that brings it in.
__device__ __forceinline__ unsigned char *place(unsigned char *&cur, const void *gbase, int64_t a, int64_t b, int e,
                                                uintptr_t *dst, uintptr_t *src, uint32_t *bytes) {
    const uintptr_t g0 = (uintptr_t)gbase + (uintptr_t)(a * e);
    const uintptr_t g1 = (uintptr_t)gbase + (uintptr_t)(b * e);
    const uintptr_t A = g0 & ~(uintptr_t)15;
    const uintptr_t B = (g1 + 15) & ~(uintptr_t)15;
    unsigned char *d = cur;
    cur += span16(b - a, e);
    *dst = (uintptr_t)d;
    *src = A;
    *bytes = (b > a) ? (uint32_t)(B - A) : 0u;
    return d + (g0 - A);
}

// One copy per lane (any lane may have none): copies up to kChunk bytes are
// issued by their own lane, larger ones split into kChunk pieces spread over
// the warp (many mid-sized bulk copies in flight move data faster than a few
// large ones).  Returns this lane's bytes.
__device__ __forceinline__ uint32_t issue_copy(uintptr_t dst, uintptr_t src, uint32_t nb, uint64_t *bar) {
    const int lane = threadIdx.x & 31;
    if (nb != 0 && nb <= kChunk) bulk_g2s((void *)dst, (const void *)src, nb, bar);
    unsigned big = __ballot_sync(0xffffffffu, nb > kChunk);
    while (big) {
        const int L = __ffs(big) - 1;
        big &= big - 1;
        const unsigned long long d = __shfl_sync(0xffffffffu, (unsigned long long)dst, L);
        const unsigned long long s = __shfl_sync(0xffffffffu, (unsigned long long)src, L);
        const uint32_t n = __shfl_sync(0xffffffffu, nb, L);
        for (uint32_t o = (uint32_t)lane * kChunk; o < n; o += 32u * kChunk)
            bulk_g2s((void *)(d + o), (const void *)(s + o), min(kChunk, n - o), bar);
    }
    return nb;
}

// exclusive warp prefix sum of each lane's level bytes: the level's offset
__device__ __forceinline__ int64_t level_offset(int64_t bytes) {
    const int lane = threadIdx.x & 31;
    int64_t off = bytes;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
    }
    return off - bytes;
}

// the warp's arrival on the unit's barrier with the total byte count; copies
// already issued may complete first, so the transaction count may go below
// zero until this arrival adds the total
__device__ __forceinline__ void arm(uint64_t *bar, uint32_t mine) {
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0) mbar_arrive_expect_tx(bar, mine);
}

// Warp 0 (all 32 lanes): lay out an up unit in buffer `buf` and start its
// copies.  Lane k < nl owns level k: it sizes the level (the same formula the
// host packer used), a warp scan places the levels one after another, and the
// lane places and issues the level's arrays one at a time.  For an internal
// unit lane nl stages the child units' top-level ev.
__device__ void issue_up(const DevPlayer &P, const int4 hdr, unsigned char *buf, uint64_t *bar, SLvl *lv,
                         UpTab *tab, ChildEv *cev) {
    const int lane = threadIdx.x & 31;
    const int32_t *rng = P.ranges + hdr.z;
    const int nl = hdr.y;
    const bool internal = (hdr.w & kInternal) != 0;
    SLvl L{0, 0, 0, 0, 0, 0};
    int64_t bytes = 0;
    if (lane < nl) {
        const int32_t *d = rng + kLvl * lane;
        L = SLvl{d[0], d[1], d[2], d[3], d[4], d[5]};
        bytes = up_level_bytes(L.s1 - L.s0, L.j1 - L.j0, L.n1 - L.n0);
    } else if (internal && lane == nl) {
        const int32_t *d = rng + kLvl * nl;
        L = SLvl{d[0], d[1], 0, 0, 0, 0};
        bytes = span16(L.j1 - L.j0, 4);
    }
    unsigned char *cur = buf + level_offset(bytes);
    fence_proxy_async();
    uint32_t mine = 0;
    const bool lvl = lane < nl;
    if (lvl) lv[lane] = L;
#pragma unroll 1
    for (int f = 0; f < 7; f++) {
        uintptr_t dst = 0, src = 0;
        uint32_t nb = 0;
        if (lvl) {
            UpTab &t = tab[lane];
            switch (f) {
            case 0: t.r = sh_off(place(cur, P.r, L.s0, L.s1, 8, &dst, &src, &nb)); break;
            case 1: t.b = sh_off(place(cur, P.b, L.s0, L.s1, 4, &dst, &src, &nb)); break;
            case 2: t.sch = sh_off(place(cur, P.seq_child, L.s0, L.s1 + 1, 4, &dst, &src, &nb)); break;
            case 3: t.mptr = sh_off(place(cur, P.m_ptr, L.s0, L.s1 + 1, 4, &dst, &src, &nb)); break;
            case 4: t.iseq = sh_off(place(cur, P.inf_seq, L.j0, L.j1 + 1, 4, &dst, &src, &nb)); break;
            case 5: t.col = sh_off(place(cur, P.m_col, L.n0, L.n1, 4, &dst, &src, &nb)); break;
            default: t.val = sh_off(place(cur, P.m_val, L.n0, L.n1, 4, &dst, &src, &nb)); break;
            }
        } else if (f == 0 && internal && lane == nl) {
            // placed now, copied once the children are done (issue_child_ev)
            cev->ev = sh_off(place(cur, P.ev, L.j0, L.j1, 4, &dst, &src, &nb));
            cev->c0 = L.j0;
            cev->dst = sh_off((const void *)dst);
            cev->bytes = nb;
            cev->src = (const void *)src;
            nb = 0;
        }
        mine += issue_copy(dst, src, nb, bar);
    }
    if (lvl) {
        tab[lane].gx = sh_off(cur);
        cur += work16(L.n1 - L.n0, 4);
        tab[lane].V = sh_off(cur);
        cur += work16(L.s1 - L.s0, 4);
        tab[lane].ev = sh_off(cur);
    }
    arm(bar, mine);
}

// One thread, once an internal unit's children are all done (acquired through
// their completion count): copy their top-level ev into the unit's buffer.
__device__ __forceinline__ void issue_child_ev(const ChildEv &c, uint64_t *bar) {
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, c.bytes);
    if (c.bytes) bulk_g2s(sh<unsigned char>(c.dst), c.src, c.bytes, bar);
}

// Warp 0: lay out a down unit in buffer `buf` and start its copies.  `what`
// selects the arrays: kDownOwn (x, xbar and the index arrays, which the
// previous kernel does not write) and/or kDownB (the strategy b the up pass
// just wrote).  The call that issues b arms the barrier with `carried` plus
// its own bytes; the return value is this lane's bytes when b is not issued.
constexpr int kDownOwn = 1, kDownB = 2;
__device__ uint32_t issue_down(const DevPlayer &P, const int4 hdr, unsigned char *buf, uint64_t *bar, SLvl *lv,
                               DownTab *tab, int what, uint32_t carried) {
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
    unsigned char *cur = buf + level_offset(bytes);
    fence_proxy_async();
    uint32_t mine = carried;
    const bool lvl = lane < nl;
    if (lvl) lv[lane] = L;
#pragma unroll 1
    for (int f = 0; f < 5; f++) {
        uintptr_t dst = 0, src = 0;
        uint32_t nb = 0;
        if (lvl) {
            DownTab &t = tab[lane];
            switch (f) {
            case 0: t.b = sh_off(place(cur, P.b, L.s0, L.s1, 4, &dst, &src, &nb)); break;
            case 1: t.x = sh_off(place(cur, P.x, L.s0, L.s1, 4, &dst, &src, &nb)); break;
            case 2: t.xbar = sh_off(place(cur, P.xbar, L.s0, L.s1, 8, &dst, &src, &nb)); break;
            case 3: t.ipar = sh_off(place(cur, P.inf_par, L.j0, L.j1, 4, &dst, &src, &nb)); break;
            default: t.iseq = sh_off(place(cur, P.inf_seq, L.j0, L.j1 + 1, 4, &dst, &src, &nb)); break;
            }
        }
        if (!(what & (f == 0 ? kDownB : kDownOwn))) nb = 0;
        mine += issue_copy(dst, src, nb, bar);
    }
    if (what & kDownB) {
        arm(bar, mine);
        return 0;
    }
    return mine;
}

// Up pass of a staged unit (consumer warps only): gathers of the other
// player's x, payoff rows, bottom-up values, regret update, variant post-op
// and next strategy, all in shared memory; then write-back.  An internal unit's deepest level finds its
// children's ev in the staged child range.  The game's root unit also runs
// its top-down pass with the new strategy (x of its sequences into xn), so
// the top-down pass below it need not wait for it.
constexpr int kRegA = 4;    // infosets with at most kRegA actions keep their values in registers

// shared-memory views of one staged up level
struct UpView {
    float2 *r;
    float *b, *V, *ev;
    const int32_t *sch, *mptr, *iseq, *col;
    float *val;
};
__device__ __forceinline__ UpView view(const UpTab &t) {
    return UpView{sh<float2>(t.r), sh<float>(t.b), sh<float>(t.V), sh<float>(t.ev), sh<const int32_t>(t.sch),
                  sh<const int32_t>(t.mptr), sh<const int32_t>(t.iseq), sh<const int32_t>(t.col), sh<float>(t.val)};
}

// One infoset i with na <= kRegA actions, in registers: V of its sequences
// (payoff row sum in CSR order, each product rounded before it is added, then
// the child ev in child order; the actions' loops interleaved), ev, regret
// update, post-op and regret matching.
struct LevelIn {
    const float *val, *gx, *evc;
    int n0, cj0;
    float sign;
    bool kids;
};
__device__ __forceinline__ void up_step_reg(const UpView &t, const LevelIn &in, int i, int q0, int na, int variant,
                                            bool pred, const ItemParams &ip) {
    float V[kRegA], bb[kRegA], qv[kRegA];
    float2 rr[kRegA];
    int e[kRegA], e1[kRegA];
    int len = 0;
#pragma unroll
    for (int a = 0; a < kRegA; a++) {
        V[a] = 0.f;
        e[a] = e1[a] = 0;
        if (a < na) {
            e[a] = t.mptr[q0 + a] - in.n0;
            e1[a] = t.mptr[q0 + a + 1] - in.n0;
            len = max(len, e1[a] - e[a]);
            bb[a] = t.b[q0 + a];
            rr[a] = t.r[q0 + a];
        }
    }
    for (int k = 0; k < len; k++) {
#pragma unroll
        for (int a = 0; a < kRegA; a++)
            if (e[a] + k < e1[a]) V[a] = __fadd_rn(V[a], __fmul_rn(in.val[e[a] + k], in.gx[e[a] + k]));
    }
#pragma unroll
    for (int a = 0; a < kRegA; a++) V[a] *= in.sign;
    if (in.kids) {
        len = 0;
#pragma unroll
        for (int a = 0; a < kRegA; a++) {
            e[a] = e1[a] = 0;
            if (a < na) {
                e[a] = t.sch[q0 + a] - in.cj0;
                e1[a] = t.sch[q0 + a + 1] - in.cj0;
                len = max(len, e1[a] - e[a]);
            }
        }
        for (int k = 0; k < len; k++) {
#pragma unroll
            for (int a = 0; a < kRegA; a++)
                if (e[a] + k < e1[a]) V[a] += in.evc[e[a] + k];
        }
    }
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
    const float inv = pos > 0.f ? __frcp_rn(pos) : 0.f;   // = 1/pos correctly rounded
    const float uni = __frcp_rn((float)na);
#pragma unroll
    for (int a = 0; a < kRegA; a++)
        if (a < na) {
            t.b[q0 + a] = pos > 0.f ? qv[a] * inv : uni;
            t.V[q0 + a] = V[a];   // kept for the root's top-down pass (overwritten there)
        }
}

// the same for infosets with more actions, through shared memory
__device__ __noinline__ void up_step_wide(UpTab tt, LevelIn in, int i, int q0, int q1, int variant, bool pred,
                                          ItemParams ip) {
    const UpView t = view(tt);
    for (int q = q0; q < q1; q++) {
        float acc = 0.f;
        for (int e = t.mptr[q] - in.n0; e < t.mptr[q + 1] - in.n0; e++)
            acc = __fadd_rn(acc, __fmul_rn(in.val[e], in.gx[e]));
        float v = in.sign * acc;
        if (in.kids)
            for (int c = t.sch[q] - in.cj0; c < t.sch[q + 1] - in.cj0; c++) v += in.evc[c];
        t.V[q] = v;
    }
    float ev = 0.f;
    for (int q = q0; q < q1; q++) ev = fmaf(t.b[q], t.V[q], ev);
    t.ev[i] = ev;
    float pos = 0.f;
    for (int q = q0; q < q1; q++) {
        const float d = t.V[q] - ev;
        float2 r = ff_add_f(t.r[q], d);
        r = post_op(r, variant, ip);
        t.r[q] = r;
        const float rr = pred ? r.x + d : r.x;
        const float qq = rr > 0.f ? rr : 0.f;
        t.V[q] = qq;   // V is no longer needed: keep the clipped regret
        pos += qq;
    }
    const float inv = pos > 0.f ? __frcp_rn(pos) : 0.f;
    const float uni = __frcp_rn((float)(q1 - q0));
    for (int q = q0; q < q1; q++) t.b[q] = pos > 0.f ? t.V[q] * inv : uni;
}

// the root's next x, top-down, into each level's V (no longer needed); level
// 0's parent is the empty sequence (x = 1)
__device__ __noinline__ void root_topdown(int nl, const SLvl *lv, const UpTab *tab) {
    const int tid = threadIdx.x - kProducerThreads, nt = blockDim.x - kProducerThreads;
    for (int k = 0; k < nl; k++) {
        const SLvl L = lv[k];
        const UpView t = view(tab[k]);
        const int ni = L.j1 - L.j0;
        for (int i = tid; i < ni; i += nt) {
            float xp = 1.f;
            if (k > 0) {
                // the parent sequence: the one of level k-1 whose child range
                // holds infoset j (child ranges are ascending)
                const UpView pt = view(tab[k - 1]);
                const int j = L.j0 + i;
                int lo = 0, hi = lv[k - 1].s1 - lv[k - 1].s0;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (pt.sch[mid] <= j) lo = mid;
                    else hi = mid;
                }
                xp = pt.V[lo];
            }
            for (int q = t.iseq[i] - L.s0; q < t.iseq[i + 1] - L.s0; q++) t.V[q] = xp * t.b[q];
        }
        consumer_sync();
    }
}

__device__ void compute_up(const DevPlayer &P, const float *__restrict__ xo, const IterArgs &ia,
                           const ItemParams &ip, int nl, const SLvl *lv, const UpTab *tab, const ChildEv *cev,
                           bool internal, bool root) {
    const int tid = threadIdx.x - kProducerThreads, nt = blockDim.x - kProducerThreads;
    // the other player's x at every payoff entry's column, gathered with
    // 4-byte asynchronous copies: every load of the unit in flight at once,
    // none of them holding a register
    for (int k = 0; k < nl; k++) {
        const int nz = lv[k].n1 - lv[k].n0;
        const int32_t *col = sh<const int32_t>(tab[k].col);
        const uint32_t gx = smem_addr(sh<float>(tab[k].gx));
#pragma unroll 4
        for (int e = tid; e < nz; e += nt) cp_async4(gx + 4u * (uint32_t)e, xo + col[e]);
    }
    cp_async_wait_all();
    consumer_sync();
    const bool pred = (ia.variant == VAR_PCFR_PLUS);
    for (int k = nl - 1; k >= 0; k--) {
        const SLvl L = lv[k];
        const UpView t = view(tab[k]);
        const int ni = L.j1 - L.j0;
        // children of this level: the unit's next level, or (an internal
        // unit's deepest level) the staged child units' top levels
        const bool deepest = (k + 1 == nl);
        LevelIn in;
        in.val = sh<const float>(tab[k].val);
        in.gx = sh<const float>(tab[k].gx);
        in.evc = sh<const float>(deepest ? cev->ev : tab[k + 1].ev);
        in.n0 = L.n0;
        in.cj0 = deepest ? cev->c0 : lv[k + 1].j0;
        in.sign = ia.sign;
        in.kids = !deepest || internal;
        for (int i = tid; i < ni; i += nt) {
            const int q0 = t.iseq[i] - L.s0, q1 = t.iseq[i + 1] - L.s0;
            if (q1 - q0 <= kRegA) up_step_reg(t, in, i, q0, q1 - q0, ia.variant, pred, ip);
            else up_step_wide(tab[k], in, i, q0, q1, ia.variant, pred, ip);
        }
        consumer_sync();
    }
    if (root) root_topdown(nl, lv, tab);
    // write-back (coalesced)
    for (int k = 0; k < nl; k++) {
        const SLvl L = lv[k];
        const UpView t = view(tab[k]);
        const int ns = L.s1 - L.s0;
        for (int q = tid; q < ns; q += nt) {
            P.r[L.s0 + q] = t.r[q];
            P.b[L.s0 + q] = t.b[q];
            if (root) P.xn[L.s0 + q] = t.V[q];
        }
    }
    if (nl > 0) {
        const int ni = lv[0].j1 - lv[0].j0;
        const float *ev = sh<const float>(tab[0].ev);
        for (int i = tid; i < ni; i += nt) P.ev[lv[0].j0 + i] = ev[i];
    }
}

// Down pass of a staged unit: x[(j,a)] = x[p_j] b_j[a] top-down, and
// xbar += w x for the strategy being replaced.  The top level's parents
// belong to the root or to internal units, whose next x the bottom-up pass
// published in xn; the roots' parent is the empty sequence (x = 1).
__device__ void compute_down(const DevPlayer &P, const IterArgs &ia, const ItemParams &ip, int nl, const SLvl *lv,
                             const DownTab *tab) {
    const int tid = threadIdx.x - kProducerThreads, nt = blockDim.x - kProducerThreads;
    const bool avg = ia.average != 0;
    const float *xtop = P.xn;
    for (int k = 0; k < nl; k++) {
        const SLvl L = lv[k];
        const DownTab t = tab[k];
        const float *b = sh<const float>(t.b);
        float *x = sh<float>(t.x);
        float2 *xbar = sh<float2>(t.xbar);
        const int32_t *ipar = sh<const int32_t>(t.ipar), *iseq = sh<const int32_t>(t.iseq);
        const int ni = L.j1 - L.j0;
        const int ps0 = (k > 0) ? lv[k - 1].s0 : 0;
        const float *xpar = (k > 0) ? sh<const float>(tab[k - 1].x) : nullptr;
        for (int i = tid; i < ni; i += nt) {
            const int par = ipar[i];
            const float xp = par < 0 ? 1.f : (k == 0 ? __ldcg(&xtop[par]) : xpar[par - ps0]);
            for (int q = iseq[i] - L.s0; q < iseq[i + 1] - L.s0; q++) {
                if (avg) xbar[q] = ff_add(xbar[q], ff_mul_f(ip.w, x[q]));
                x[q] = xp * b[q];
            }
        }
        consumer_sync();
    }
    for (int k = 0; k < nl; k++) {
        const SLvl L = lv[k];
        const float *x = sh<const float>(tab[k].x);
        const float2 *xbar = sh<const float2>(tab[k].xbar);
        const int ns = L.s1 - L.s0;
        for (int q = tid; q < ns; q += nt) {
            P.x[L.s0 + q] = x[q];
            if (avg) P.xbar[L.s0 + q] = xbar[q];
        }
    }
}

}  // namespace cfrb
