// Shared-memory staged units for the two per-player passes.
//
// A unit (layout.h) is one contiguous range per level of every array it
// touches, so the producer warp can copy the whole unit into shared memory
// with bulk asynchronous copies (cp.async.bulk, completion counted in bytes on
// an mbarrier) before any index is read.  The consumer warps then run the
// unit's levels out of shared memory: the bottom-up steps store their results
// (r, b, ev) straight to global memory, the top-down pass writes its own
// levels' x back with coalesced stores.  Two buffers per CTA: the next unit's
// copies are in flight while the current one is computed, and several CTAs
// share an SM.
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace cfrb {

constexpr uint32_t kWaitLimit = 1u << 26;          // polls of an mbarrier before giving up
constexpr uint64_t kFlagWaitNs = 1000000000ull;    // default longest wait for another unit (1 s)
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
// the same for shared memory only: a buffer's earlier generic accesses come
// before the bulk copies that refill it
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s_to(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
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
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
// 16 bytes, through L2 only (data another SM wrote: no stale L1 line)
__device__ __forceinline__ void cp_async16_cg_to(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16_cg(void *dst, const void *src) { cp_async16_cg_to(smem_addr(dst), src); }
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
// if it does not happen within limit_ns.  The poll interval stays short: only
// one thread of a waiting CTA polls, and a waiting unit is on the pass's
// critical path (a longer sleep only delays its wake-up).
__device__ __forceinline__ bool flag_wait(const int32_t *flag, int want, int32_t *err, uint64_t limit_ns) {
    if (ld_acquire(flag) == want) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t k = 0;; k++) {
        __nanosleep(32);
        if (ld_acquire(flag) == want) return true;
        if ((k & 15) == 15 && globaltimer() - t0 > limit_ns) break;
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
    uint32_t gx;    // the other player's x: per payoff entry (gathered), or nwin copied windows
    int32_t nwin;   // 0: gathered per entry
    uint32_t V;     // float counterfactual values, then clipped regrets, then (root) next x
    uint32_t ev;    // float ev per infoset
};
struct DownTab {
    uint32_t b;     // float, copied in
    uint32_t x;     // float, the next x: computed in place over b (each sequence's b is read
                    // once, by the thread that then writes its x)
    uint32_t ipar, iseq;
};
constexpr int kDownArrays = 3;   // commands staged per top-down level: b, infoset parents, infoset segments
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
    __syncwarp();   // the lanes' layout writes (lv, tab) come before the arrival (release)
    if ((threadIdx.x & 31) == 0) mbar_arrive_expect_tx(bar, mine);
}

// Warp 0 (all 32 lanes): lay out an up unit in buffer `buf` and start its
// copies.  Lane k < nl owns level k: it sizes the level (the same formula the
// host packer used), a warp scan places the levels one after another, and the
// lane places and issues the level's arrays one at a time.  For an internal
// unit lane nl stages the child units' top-level ev.
// One bulk copy global -> shared, as staged by the producer before issue.
struct BulkCmd {
    const void *src;
    uint32_t dst;     // shared address
    uint32_t bytes;
};
constexpr int kUpArrays = 7;   // arrays staged per up level

// What the producer needs to lay out and issue one up unit, copied into
// shared memory a round before the unit is issued, so that issuing reads no
// global memory: the queue entry, the unit's parameters, each level's range
// record and window record, an internal unit's child range, and the unit's
// first kPreWin x windows.
constexpr int kPreWin = 64;
struct __align__(16) UpPre {
    int4 h, q;            // queue entry: {game, nlvl, rng, flags | nwin << 8}, {unit, parent, nchild, W0}
    ItemParams ip;
    int4 xw[kMaxStagedLevels];   // per level: {w0, w1, x-area bytes, 0}
    int4 win[kPreWin];    // {c0, c1, byte offset, level}
    SLvl lv[kMaxStagedLevels];
    int2 child;           // internal unit: the child units' top-level infosets
    int32_t pos;          // queue position; n: none
};
static_assert(sizeof(ItemParams) == 32, "ItemParams is copied as two 16-byte pieces");
__device__ __forceinline__ int unit_nwin(const int4 h) { return h.w >> 8; }

// Warp 0 (all lanes): start copying the records of the up unit at queue
// position pos (< n), whose queue entry {h, q} is at hand, into `pre` with
// asynchronous copies; they land while the producer goes on (the next
// cp.async.wait_all of these lanes waits for them).  Range records are
// 8-byte aligned (every record starts at an even int), the others 16.
__device__ void up_prefetch(const DevPlayer &P, const DevGames &gm, const IterArgs &ia, int pos, int4 h, int4 q,
                            UpPre &pre) {
    const int lane = threadIdx.x & 31;
    const int nl = h.y;
    if (lane < nl) {
        const int32_t *d = P.ranges + h.z + kLvl * lane;
        int32_t *o = &pre.lv[lane].j0;
        cp_async8(o, d);
        cp_async8(o + 2, d + 2);
        cp_async8(o + 4, d + 4);
        cp_async16(&pre.xw[lane], &P.rwin[h.z / kLvl + lane]);
    } else if (lane == nl && (h.w & kInternal)) {
        cp_async8(&pre.child, P.ranges + h.z + kLvl * nl);
    } else if (lane == 30 || lane == 31) {
        const ItemParams *src = &gm.par[(int64_t)h.x * (kParamSpan + 1) + ia.pslot];
        cp_async16((char *)&pre.ip + 16 * (lane - 30), (const char *)src + 16 * (lane - 30));
    }
    const int nw = min(unit_nwin(h), kPreWin);
    for (int w = lane; w < nw; w += 32) cp_async16(&pre.win[w], &P.win[q.w + w]);
    if (lane == 0) {
        pre.h = h;
        pre.q = q;
        pre.pos = pos;
    }
}

// Warp 0 (all lanes): the x windows of a staged unit, one window per lane,
// each into its level's x area at its offset (the layout, tab[k].gx, is this
// warp's own work, made visible by __syncwarp).  Windows past the prefetched
// ones come from global memory.  Issues the copies when `issue`; returns this
// lane's bytes either way.
__device__ __forceinline__ uint32_t issue_windows(const DevPlayer &P, const float *__restrict__ xo, const int4 h,
                                                  const int4 q, const int4 *prewin, const UpTab *tab, uint64_t *bar,
                                                  bool issue) {
    __syncwarp();
    uint32_t mine = 0;
    const int nw = unit_nwin(h);
    for (int w = (int)(threadIdx.x & 31); w < nw; w += 32) {
        const int4 d = (prewin && w < kPreWin) ? prewin[w] : P.win[q.w + w];   // {c0, c1, byte offset, level}
        unsigned char *cur = sh<unsigned char>(tab[d.w].gx) + d.z;
        uintptr_t dst = 0, src = 0;
        uint32_t nb = 0;
        place(cur, xo, d.x, d.y, 4, &dst, &src, &nb);
        if (issue && nb) bulk_g2s((void *)dst, (const void *)src, nb, bar);
        mine += nb;
    }
    return mine;
}

// The x windows of a unit laid out by issue_up with `defer_x`, once the
// other player's x may be read (the previous kernel is done): thread t of nt
// copies its 16-byte pieces of each window (d: the unit's window records).
__device__ void copy_up_x(const float *__restrict__ xo, int nw, const int4 *d, const UpTab *tab, int t, int nt) {
    for (int w = 0; w < nw; w++) {
        unsigned char *cur = sh<unsigned char>(tab[d[w].w].gx) + d[w].z;
        uintptr_t dst = 0, src = 0;
        uint32_t nb = 0;
        place(cur, xo, d[w].x, d[w].y, 4, &dst, &src, &nb);
        for (uint32_t k = 16u * (uint32_t)t; k < nb; k += 16u * (uint32_t)nt)
            cp_async16_cg((void *)(dst + k), (const void *)(src + k));
    }
}

// Warp 0 (all lanes): lay out the prefetched up unit in buffer `buf` and
// start its copies.  Lane k < nl owns level k: it sizes the level (the same
// formula the host packer used), a warp scan places the levels one after
// another, and the lane places and issues the level's arrays one at a time.
// For an internal unit lane nl places the child units' top-level ev.
__device__ void issue_up(const DevPlayer &P, const float *__restrict__ xo, const UpPre &pre, unsigned char *buf,
                         uint64_t *bar, SLvl *lv, UpTab *tab, ChildEv *cev, BulkCmd *cmd, bool defer_x) {
    const int lane = threadIdx.x & 31;
    const int4 hdr = pre.h;
    const int nl = hdr.y;
    const bool internal = (hdr.w & kInternal) != 0;
    SLvl L{0, 0, 0, 0, 0, 0};
    int64_t bytes = 0;
    int2 xb = make_int2(0, 0);   // x-area bytes, x windows (0: gathered)
    if (lane < nl) {
        L = pre.lv[lane];
        const int4 r = pre.xw[lane];
        xb = make_int2(r.z, r.y - r.x);
        bytes = up_level_bytes_x(L.s1 - L.s0, L.j1 - L.j0, L.n1 - L.n0, xb.x);
    } else if (internal && lane == nl) {
        L = SLvl{pre.child.x, pre.child.y, 0, 0, 0, 0};
        bytes = span16(L.j1 - L.j0, 4);
    }
    unsigned char *cur = buf + level_offset(bytes);
    fence_proxy_async_smem();
    // placement: each level's lane lays out its arrays and stages their
    // copies as commands
    if (lane < nl) {
        lv[lane] = L;
        UpTab &t = tab[lane];
        BulkCmd *c = cmd + kUpArrays * lane;
        uintptr_t dst = 0, src = 0;
        uint32_t nb = 0;
#define CFR_STAGE(field, arr, a, b, e, f)                                     \
    t.field = sh_off(place(cur, arr, a, b, e, &dst, &src, &nb));             \
    c[f] = BulkCmd{(const void *)src, smem_addr((const void *)dst), nb};
        CFR_STAGE(r, P.r, L.s0, L.s1, 8, 0)
        CFR_STAGE(b, P.b, L.s0, L.s1, 4, 1)
        CFR_STAGE(sch, P.seq_child, L.s0, L.s1 + 1, 4, 2)
        CFR_STAGE(mptr, P.m_ptr, L.s0, L.s1 + 1, 4, 3)
        CFR_STAGE(iseq, P.inf_seq, L.j0, L.j1 + 1, 4, 4)
        CFR_STAGE(col, P.lcol, L.n0, L.n1, 4, 5)
        CFR_STAGE(val, P.m_val, L.n0, L.n1, 4, 6)
#undef CFR_STAGE
        t.gx = sh_off(cur);
        t.nwin = xb.y;
        cur += xb.x;
        t.V = sh_off(cur);
        cur += work16(L.s1 - L.s0, 4);
        t.ev = sh_off(cur);
    } else if (internal && lane == nl) {
        // placed now, copied once the children are done (copy_child_ev)
        uintptr_t dst = 0, src = 0;
        uint32_t nb = 0;
        cev->ev = sh_off(place(cur, P.ev, L.j0, L.j1, 4, &dst, &src, &nb));
        cev->c0 = L.j0;
        cev->dst = sh_off((const void *)dst);
        cev->bytes = nb;
        cev->src = (const void *)src;
    }
    __syncwarp();
    // issue: one command per lane, all lanes at once (larger copies in
    // kChunk pieces by their lane)
    uint32_t mine = 0;
    for (int k = lane; k < kUpArrays * nl; k += 32) {
        const BulkCmd c = cmd[k];
        for (uint32_t o = 0; o < c.bytes; o += kChunk)
            bulk_g2s_to(c.dst + o, (const char *)c.src + o, min(kChunk, c.bytes - o), bar);
        mine += c.bytes;
    }
    // deferred windows are copied by the whole CTA later, outside the barrier
    if (unit_nwin(hdr) > 0 && !defer_x) mine += issue_windows(P, xo, hdr, pre.q, pre.win, tab, bar, true);
    arm(bar, mine);
}

// Once an internal unit's children are all done (acquired through their
// completion count): consumer thread t of nt copies its 16-byte pieces of the
// children's top-level ev into the unit's buffer.
__device__ __forceinline__ void copy_child_ev(const ChildEv &c, int t, int nt) {
    for (uint32_t k = 16u * (uint32_t)t; k < c.bytes; k += 16u * (uint32_t)nt)
        cp_async16_cg(sh<unsigned char>(c.dst) + k, (const unsigned char *)c.src + k);
}

// Warp 0: lay out a down unit in buffer `buf` (its ancestor chain first, then
// its own levels), stage its copies as commands (cmd[kDownArrays * level + f]:
// f = 0 b, 1 infoset parents, 2 infoset segments) and issue those `what`
// selects: kDownOwn (the index arrays, which no pass writes) and/or kDownB
// (b, which the bottom-up pass writes).  With kDownArm the barrier is armed
// with `carried` plus the bytes issued here.  Returns this lane's bytes.
constexpr int kDownOwn = 1, kDownB = 2, kDownArm = 4;
__device__ uint32_t issue_down(const DevPlayer &P, const int4 hdr, unsigned char *buf, uint64_t *bar, SLvl *lv,
                               DownTab *tab, BulkCmd *cmd, int what, uint32_t carried) {
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
    // placement by each level's lane, copies staged as commands
    if (lane < nl) {
        lv[lane] = L;
        DownTab &t = tab[lane];
        BulkCmd *c = cmd + kDownArrays * lane;
        uintptr_t dst = 0, src = 0;
        uint32_t nb = 0;
#define CFR_STAGE(field, arr, a, b, e, f)                                        \
    t.field = sh_off(place(cur, arr, a, b, e, &dst, &src, &nb));                \
    c[f] = BulkCmd{(const void *)src, smem_addr((const void *)dst), nb};
        CFR_STAGE(b, P.b, L.s0, L.s1, 4, 0)
        CFR_STAGE(ipar, P.inf_par, L.j0, L.j1, 4, 1)
        CFR_STAGE(iseq, P.inf_seq, L.j0, L.j1 + 1, 4, 2)
#undef CFR_STAGE
        t.x = t.b;
    }
    __syncwarp();
    uint32_t mine = carried;
    for (int k = lane; k < kDownArrays * nl; k += 32) {
        const int f = k % kDownArrays;
        if (!(what & (f == 0 ? kDownB : kDownOwn))) continue;
        const BulkCmd c = cmd[k];
        for (uint32_t o = 0; o < c.bytes; o += kChunk)
            bulk_g2s_to(c.dst + o, (const char *)c.src + o, min(kChunk, c.bytes - o), bar);
        mine += c.bytes;
    }
    if (what & kDownArm) arm(bar, mine);
    return mine;
}

// Up pass of a staged unit (consumer warps only): gathers of the other
// player's x, payoff rows, bottom-up values, regret update, variant post-op
// and next strategy, all out of shared memory; each step stores its new r, b
// (and the ev its parent reads) to global memory.  An internal unit's deepest
// level finds its children's ev in the staged child range.
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

// The staged bottom-up work of one level is split into phases, each a short
// chain per thread, so that no thread walks a long data-dependent loop (a
// shared-memory load is ~30-50 cycles, and a warp waits for its longest lane):
//   rows:  V[s] = sign * (sum of the payoff products of row s, in CSR order),
//          one thread per sequence, every level of the unit at once;
//   kids:  V[s] += ev of each child infoset, in child order, one thread per
//          sequence (the levels below are done);
//   step:  one thread per infoset: ev = sum_a b[a] V[a], the regret update and
//          post-op, regret matching (straight-line code for <= kRegA actions).
// Every sum runs in the same order as in the global-memory path, so results
// do not depend on how a game is cut into units.  The step stores the new r
// and b straight to global memory (gr, gb: the level's first sequence) and,
// when gev is given, ev too (the level's first infoset); the staged ev stays
// in shared memory for the level above.
template <int VAR>
__device__ __forceinline__ void up_step_reg(const UpView &t, int i, int q0, int na, float2 fpos, float2 fneg,
                                            float2 *gr, float *gb, float *gev) {
    float V[kRegA], bb[kRegA];
    float2 rr[kRegA];
#pragma unroll
    for (int a = 0; a < kRegA; a++) {
        const int q = q0 + min(a, na - 1);   // past the last action: a repeat, unused
        V[a] = t.V[q];
        bb[a] = t.b[q];
        rr[a] = t.r[q];
    }
    float ev = 0.f;
#pragma unroll
    for (int a = 0; a < kRegA; a++)
        if (a < na) ev = fmaf(bb[a], V[a], ev);
    t.ev[i] = ev;
    if (gev) gev[i] = ev;
    float pos = 0.f, qv[kRegA];
#pragma unroll
    for (int a = 0; a < kRegA; a++) {
        const float d = V[a] - ev;
        const float2 r = post_op_v<VAR>(ff_add_f(rr[a], d), fpos, fneg);
        if (a < na) gr[q0 + a] = r;
        const float x = predictive(VAR) ? r.x + d : r.x;
        qv[a] = (a < na && x > 0.f) ? x : 0.f;
        pos += qv[a];
    }
    const RmNorm nrm = rm_norm(pos);
    const float uni = uniform_prob(na);
#pragma unroll
    for (int a = 0; a < kRegA; a++)
        if (a < na) gb[q0 + a] = pos > 0.f ? rm_prob(qv[a], nrm) : uni;
}

// the same for infosets with more actions, through shared memory
template <int VAR>
__device__ __noinline__ void up_step_wide(UpTab tt, int i, int q0, int q1, float2 fpos, float2 fneg, float2 *gr,
                                          float *gb, float *gev) {
    const UpView t = view(tt);
    float ev = 0.f;
    for (int q = q0; q < q1; q++) ev = fmaf(t.b[q], t.V[q], ev);
    t.ev[i] = ev;
    if (gev) gev[i] = ev;
    float pos = 0.f;
    for (int q = q0; q < q1; q++) {
        const float d = t.V[q] - ev;
        const float2 r = post_op_v<VAR>(ff_add_f(t.r[q], d), fpos, fneg);
        gr[q] = r;
        const float rr = predictive(VAR) ? r.x + d : r.x;
        const float qq = rr > 0.f ? rr : 0.f;
        t.V[q] = qq;   // V is no longer needed: keep the clipped regret
        pos += qq;
    }
    const RmNorm nrm = rm_norm(pos);
    const float uni = uniform_prob(q1 - q0);
    for (int q = q0; q < q1; q++) gb[q] = pos > 0.f ? rm_prob(t.V[q], nrm) : uni;
}

// Ordered sums over a short index range, four terms per step: the four
// terms' loads are issued together (indices past the end are clamped, their
// terms skipped), then added in index order, so the result is that of the
// plain left-to-right loop.  term(i) returns the i-th term.
template <class T>
__device__ __forceinline__ float ordered_sum(float acc, int i0, int i1, T &&term) {
    for (int i = i0; i < i1; i += 4) {
        float t[4];
#pragma unroll
        for (int k = 0; k < 4; k++) t[k] = term(min(i + k, i1 - 1));
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (i + k < i1) acc = __fadd_rn(acc, t[k]);
    }
    return acc;
}

// the levels of a staged unit, bottom-up, for one variant (the rows are done)
template <int VAR>
__device__ __forceinline__ void up_levels(const DevPlayer &P, const ItemParams &ip, float sign, int nl,
                                          const SLvl *lv, const UpTab *tab, const ChildEv *cev, bool internal,
                                          bool all_ev) {
    const int tid = threadIdx.x - kProducerThreads, nt = blockDim.x - kProducerThreads;
    const float2 fpos = ip.fpos, fneg = ip.fneg;
    for (int k = nl - 1; k >= 0; k--) {
        const SLvl L = lv[k];
        const UpView t = view(tab[k]);
        // children of this level: the unit's next level, or (an internal
        // unit's deepest level) the staged child units' top levels
        const bool deepest = (k + 1 == nl);
        if (!deepest || internal) {
            const float *evc = sh<const float>(deepest ? cev->ev : tab[k + 1].ev);
            const int cj0 = deepest ? cev->c0 : lv[k + 1].j0;
            const int ns = L.s1 - L.s0;
            // a level without payoff entries had no row pass: its rows are
            // sign * 0, the value the row pass gives an empty row
            const bool rows = L.n1 > L.n0;
            for (int q = tid; q < ns; q += nt)
                t.V[q] = ordered_sum(rows ? t.V[q] : sign * 0.f, t.sch[q] - cj0, t.sch[q + 1] - cj0,
                                     [&](int c) { return evc[c]; });
            consumer_sync();
        }
        const int ni = L.j1 - L.j0;
        float2 *gr = P.r + L.s0;
        float *gb = P.b + L.s0;
        float *gev = (k == 0 || all_ev) ? P.ev + L.j0 : nullptr;   // the parent reads the top level's
        for (int i = tid; i < ni; i += nt) {
            const int q0 = t.iseq[i] - L.s0, q1 = t.iseq[i + 1] - L.s0;
            if (q1 - q0 <= kRegA) up_step_reg<VAR>(t, i, q0, q1 - q0, fpos, fneg, gr, gb, gev);
            else up_step_wide<VAR>(tab[k], i, q0, q1, fpos, fneg, gr, gb, gev);
        }
        consumer_sync();
    }
}

// The payoff rows of a staged unit are worked by one consumer thread per
// sequence, every level of the unit in one numbering (the thread index runs on
// across levels, so a short level does not idle a round).  f(k, q) is called
// for level k, sequence q of the level, by the thread that owns it.  A level
// without payoff entries is skipped, except a leaf's deepest level (no child
// phase follows it there): its values start at sign * 0 in the child phase.
__device__ __forceinline__ bool level_has_rows(const SLvl *lv, int k, int nl, bool internal) {
    return lv[k].n1 > lv[k].n0 || (k + 1 == nl && !internal);
}
template <class F>
__device__ __forceinline__ void for_rows(int nl, const SLvl *lv, bool internal, F &&f) {
    const int tid = threadIdx.x - kProducerThreads, nt = blockDim.x - kProducerThreads;
    int off = 0;
    for (int k = 0; k < nl; k++) {
        if (!level_has_rows(lv, k, nl, internal)) continue;
        const int ns = lv[k].s1 - lv[k].s0;
        int q = tid - off;
        if (q < 0) q += nt;
        for (; q < ns; q += nt) f(k, q);
        off = (off + ns) % nt;
    }
}

// Up pass of a staged unit, part 1 (consumer warps): the other player's x at
// every payoff entry's column, gathered with 4-byte asynchronous copies, each
// row's by the thread that will sum it.  Issued as soon as the unit's arrays
// are in, which is normally while the previous unit is still being written
// back, so the gathers' latency is hidden.
__device__ __forceinline__ void up_gather(const float *__restrict__ xo, int nl, const SLvl *lv, const UpTab *tab,
                                          bool internal) {
    for_rows(nl, lv, internal, [&](int k, int q) {
        if (tab[k].nwin) return;   // copied in as windows
        const int n0 = lv[k].n0;
        const int32_t *mptr = sh<const int32_t>(tab[k].mptr);
        const int32_t *col = sh<const int32_t>(tab[k].col);
        const uint32_t gx = smem_addr(sh<float>(tab[k].gx));
        const int e1 = mptr[q + 1] - n0;
        for (int e = mptr[q] - n0; e < e1; e++) cp_async4(gx + 4u * (uint32_t)e, xo + col[e]);
    });
}

// Part 2: the row sums V[s] = sign * sum_e val[e] x[col[e]] (products rounded,
// then added in CSR order), each by the thread that gathered the row (its
// own copies are complete, no barrier needed); then the levels bottom-up,
// whose steps store r, b and ev to global memory.
__device__ void compute_up(const DevPlayer &P, const IterArgs &ia, const ItemParams &ip, int nl, const SLvl *lv,
                           const UpTab *tab, const ChildEv *cev, bool internal) {
    cp_async_wait_all();
    for_rows(nl, lv, internal, [&](int k, int q) {
        const int n0 = lv[k].n0;
        const int32_t *mptr = sh<const int32_t>(tab[k].mptr);
        const float *val = sh<const float>(tab[k].val);
        const float *gx = sh<const float>(tab[k].gx);
        const int e0 = mptr[q] - n0, e1 = mptr[q + 1] - n0;
        float acc;
        if (tab[k].nwin) {
            const int32_t *col = sh<const int32_t>(tab[k].col);
            acc = ordered_sum(0.f, e0, e1, [&](int e) { return __fmul_rn(val[e], gx[col[e]]); });
        } else {
            acc = ordered_sum(0.f, e0, e1, [&](int e) { return __fmul_rn(val[e], gx[e]); });
        }
        sh<float>(tab[k].V)[q] = ia.sign * acc;
    });
    consumer_sync();
    switch (ia.variant) {
    case VAR_PLUS: up_levels<VAR_PLUS>(P, ip, ia.sign, nl, lv, tab, cev, internal, ia.keep_values != 0); break;
    case VAR_DCFR: up_levels<VAR_DCFR>(P, ip, ia.sign, nl, lv, tab, cev, internal, ia.keep_values != 0); break;
    case VAR_PCFR_PLUS: up_levels<VAR_PCFR_PLUS>(P, ip, ia.sign, nl, lv, tab, cev, internal, ia.keep_values != 0); break;
    case VAR_PCFR: up_levels<VAR_PCFR>(P, ip, ia.sign, nl, lv, tab, cev, internal, ia.keep_values != 0); break;
    default: up_levels<VAR_CFR>(P, ip, ia.sign, nl, lv, tab, cev, internal, ia.keep_values != 0); break;
    }
}

// Down pass of a staged unit: x[(j,a)] = x[p_j] b_j[a] top-down over its
// levels, the first n_anc of which are its ancestor chain (down to the parents
// of its top level); level 0 of the chain holds the game's root, whose parent
// is the empty sequence (x = 1).  Only the unit's own levels are written back.
constexpr int kSoloInfosets = 64;   // ancestor levels this small are worked by one warp

__device__ void compute_down(const DevPlayer &P, int nl, int n_anc, const SLvl *lv, const DownTab *tab) {
    const int tid0 = threadIdx.x - kProducerThreads, nt0 = blockDim.x - kProducerThreads;
    bool pending = false;   // levels worked by the first consumer warp alone since the last barrier
    for (int k = 0; k < nl; k++) {
        const SLvl L = lv[k];
        const DownTab t = tab[k];
        const float *b = sh<const float>(t.b);
        float *x = sh<float>(t.x);
        const int32_t *ipar = sh<const int32_t>(t.ipar), *iseq = sh<const int32_t>(t.iseq);
        const int ni = L.j1 - L.j0;
        const int ps0 = (k > 0) ? lv[k - 1].s0 : 0;
        const float *xpar = sh<const float>((k > 0) ? tab[k - 1].x : t.x);
        // the ancestor chain is usually a few infosets per level: one warp
        // works those levels, synchronising only its lanes
        const bool solo = k < n_anc && ni <= kSoloInfosets;
        if (!solo && pending) {
            consumer_sync();
            pending = false;
        }
        if (solo && tid0 >= 32) {
            pending = true;
            continue;
        }
        const int tid = tid0, nt = solo ? 32 : nt0;
        for (int i = tid; i < ni; i += nt) {
            const int par = ipar[i];
            const float xp = par < 0 ? 1.f : xpar[par - ps0];
            // the infoset's sequences four at a time, loads first
            const int q1 = iseq[i + 1] - L.s0;
            for (int q = iseq[i] - L.s0; q < q1; q += 4) {
                float bb[4];
#pragma unroll
                for (int a = 0; a < 4; a++) bb[a] = b[min(q + a, q1 - 1)];
#pragma unroll
                for (int a = 0; a < 4; a++)
                    if (q + a < q1) x[q + a] = xp * bb[a];
            }
        }
        if (solo) {
            __syncwarp();
            pending = true;
        } else {
            consumer_sync();
        }
    }
    if (pending) consumer_sync();
    const int tid = tid0, nt = nt0;
    for (int k = n_anc; k < nl; k++) {
        const SLvl L = lv[k];
        const float *x = sh<const float>(tab[k].x);
        const int ns = L.s1 - L.s0;
        for (int q = tid; q < ns; q += nt) P.x[L.s0 + q] = x[q];
    }
}

}  // namespace cfrb
