// C ABI of the B300 CFR library: context, device buffers, kernels, CUDA graphs.
//
// Declarations and contracts: include/cfr.h.  Layout: layout.h.  Device
// building blocks: kernels.cuh (global-memory path, float-float arithmetic)
// and staged.cuh (shared-memory staged work units).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/cfr.h"
#include "kernels.cuh"
#include "layout.h"
#include "staged.cuh"

using namespace cfrb;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
namespace cfrb {

// the last CTA to leave a launch resets the queue words q = {head, exit
// count, epoch} for the next launch and advances the epoch
__device__ __forceinline__ void launch_exit(int32_t *q) {
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&q[1], 1) == (int)gridDim.x - 1) {
            q[0] = 0;
            q[1] = 0;
            atomicAdd(&q[2], 1);
        }
    }
}

// the same for the bottom-up queue and the average pass's queue at once (one
// exit count, kept in q[1]; both epochs advance)
__device__ __forceinline__ void launch_exit2(int32_t *q, int32_t *qa) {
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&q[1], 1) == (int)gridDim.x - 1) {
            q[0] = 0;
            q[1] = 0;
            qa[0] = 0;
            __threadfence();
            atomicAdd(&qa[2], 1);
            atomicAdd(&q[2], 1);
        }
    }
}

// Programmatic dependent launch: a pass may start while the previous kernel
// on the stream finishes.  pdl_wait blocks until that kernel has completed and
// its memory is visible (it returns at once for an ordinary launch);
// pdl_trigger lets the next kernel start.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Bottom-up completion of unit u (every thread of the CTA, after its
// results are written): count it at its parent.
__device__ __forceinline__ void unit_done(const DevPlayer &P, int u) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const int par = P.unit_tree[u].x;
        if (par >= 0) {
            __threadfence();
            atomicAdd(&P.unit_cnt[par], 1);
        }
    }
}

// Per-game parameters of iterations t = t_done + k, k = 0..kParamSpan, for the
// passes that follow (one thread per entry).  A game whose counter or active
// flag differs from game 0's marks the table mixed (the flag is cleared before
// the launch).
__global__ void k_params(DevGames gm, IterArgs ia, int G) {
    const int64_t n = (int64_t)G * (kParamSpan + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(e / (kParamSpan + 1)), k = (int)(e % (kParamSpan + 1));
        const int32_t t0 = gm.t_done[g];
        params_of_t(gm, ia, g, t0 + k, &gm.par[e], gm.par64 ? &gm.par64[e] : nullptr);
        if (k == 0) {
            gm.pbase[g] = t0;
            if (t0 != gm.t_done[0] || gm.active[g] != gm.active[0]) *gm.mixed = 1;
        }
    }
}

__device__ void average_pass64(const DevPlayer &P, const DevGames &gm, const IterArgs &ia, int64_t S);

// Passes over every unit from global memory, in bottom-up queue order: an
// internal unit waits (bounded) until its children are done.  MODE_BR: the
// FP64 best response (the root's ev is the game's best-response value);
// MODE_CFR64: the bottom-up pass of an FP64 iteration (precision 64), with
// the average update once the queue is empty, as in the staged pass.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_up(DevPlayer P, DevGames gm, const void *xo, IterArgs ia) {
    extern __shared__ __align__(128) unsigned char smem[];
    void *stage = smem;
    __shared__ int s_item, s_err;
    __shared__ ItemParams s_ip;
    __shared__ ItemParams64 s_ip64;
    if (threadIdx.x == 0) s_err = MODE == MODE_CFR64 && __ldcg(P.err) != 0;   // a timed-out context does no work
    __syncthreads();
    for (;;) {
        if (s_err) break;
        if (threadIdx.x == 0) s_item = atomicAdd(&P.qup[0], 1);
        __syncthreads();
        const int it = s_item;
        if (it >= P.n_up) break;
        const int4 d = P.upq[2 * it];
        const int4 q = P.upq[2 * it + 1];
        const int u = q.x;
        const int2 tr = make_int2(q.y, q.z);
        if (threadIdx.x == 0) {
            if (MODE == MODE_CFR64) {
                s_ip64 = gm.par64[(int64_t)d.x * (kParamSpan + 1) + ia.pslot];
                s_ip.active = s_ip64.active;
                s_ip.t = s_ip64.t;
            } else {
                item_params(gm, ia, d.x, &s_ip);
            }
            if (s_ip.active && tr.y > 0) {
                if (!flag_wait(&P.unit_cnt[u], tr.y, P.err, P.wait_ns)) s_err = 1;
                P.unit_cnt[u] = 0;
                __threadfence();
            }
        }
        __syncthreads();
        const ItemParams ip = s_ip;
        if (s_err) break;
        if (!ip.active) continue;
        run_up<MODE>(P, xo, ia, ip, d.y, P.ranges + d.z, stage, &s_ip64);
        unit_done(P, u);
        if (threadIdx.x == 0 && tr.x < 0 && MODE == MODE_BR) gm.br[d.x] = __ldcg(&P.ev64[d.x]);
        if (threadIdx.x == 0 && tr.x < 0 && MODE == MODE_CFR64 && ia.first_of_iter) gm.t_done[d.x] = ip.t;
    }
    if (MODE == MODE_CFR64) {
        if (ia.average && !s_err) average_pass64(P, gm, ia, P.S);
        __syncthreads();
        launch_exit2(P.qup, P.qavg);
    } else {
        launch_exit(P.qup);
    }
}

// The average strategy's update xbar += t^gamma x for the strategy x about to
// be replaced (Alg. 2; the weights of Alg. 3-5), every sequence of games that
// are advanced.  It needs only x and the iteration counter, so the bottom-up
// pass's CTAs run it once they run out of units, while the last units finish
// (the top-down pass, which overwrites x, comes after).  Chunks of kAvgChunk
// sequences are taken from a queue; the last CTA to leave resets it.
constexpr int kAvgChunk = 1024;
constexpr int kAvgU = 4;   // sequences per thread with loads in flight together
// One chunk's sequences [q0, q1).  UNIFORM: every game has game 0's
// parameters; otherwise each sequence looks up its game's weight (the
// sequences of several games are interleaved level by level), all kAvgU
// lookups of a thread in flight together.  A sequence the player does not
// reach (x = 0: regret matching gave one of its actions probability 0) adds
// exactly nothing, so its sums are neither read nor written; most sequences
// of a large game are such zeros once the regrets have settled.
template <bool UNIFORM>
__device__ __forceinline__ void average_chunk(const DevPlayer &P, const DevGames &gm, const IterArgs &ia,
                                              const ItemParams &ip0, int64_t q0, int64_t q1) {
    for (int64_t q = q0 + threadIdx.x; q < q1; q += kAvgU * blockDim.x) {
        float xv[kAvgU];
        float2 xb[kAvgU], w[kAvgU];
        int gq[kAvgU], act[kAvgU];
#pragma unroll
        for (int u = 0; u < kAvgU; u++) {
            const int64_t s = min(q + u * (int64_t)blockDim.x, q1 - 1);
            xv[u] = P.x[s];
            if (!UNIFORM) gq[u] = P.seq_game[s];
        }
#pragma unroll
        for (int u = 0; u < kAvgU; u++) {
            const int64_t s = min(q + u * (int64_t)blockDim.x, q1 - 1);
            xb[u] = xv[u] != 0.f ? P.xbar[s] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kAvgU; u++) {
            if (UNIFORM) {
                w[u] = ip0.w;
                act[u] = ip0.active;
            } else {
                const ItemParams *pp = &gm.par[(int64_t)gq[u] * (kParamSpan + 1) + ia.pslot];
                w[u] = pp->w;
                act[u] = pp->active;
            }
        }
#pragma unroll
        for (int u = 0; u < kAvgU; u++) {
            const int64_t s = q + u * (int64_t)blockDim.x;
            if (s < q1 && act[u] && xv[u] != 0.f) P.xbar[s] = ff_add(xb[u], ff_mul_f(w[u], xv[u]));
        }
    }
}

__device__ void average_pass(const DevPlayer &P, const DevGames &gm, const IterArgs &ia, int64_t S) {
    __shared__ int s_chunk;
    const int64_t nch = (S + kAvgChunk - 1) / kAvgChunk;
    // one game, or a batch advanced in step: one set of parameters
    const bool uniform = P.G == 1 || __ldcg(gm.mixed) == 0;
    const ItemParams ip0 = unit_params(gm, ia, 0);
    if (threadIdx.x == 0) s_chunk = atomicAdd(&P.qavg[0], 1);
    for (;;) {
        __syncthreads();
        const int64_t c = s_chunk;
        if (c >= nch) break;
        __syncthreads();   // s_chunk is read: the next fetch (its result lands while this chunk is worked)
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(&P.qavg[0], 1);
        const int64_t q0 = c * kAvgChunk, q1 = min((int64_t)S, q0 + kAvgChunk);
        if (uniform)
            average_chunk<true>(P, gm, ia, ip0, q0, q1);
        else
            average_chunk<false>(P, gm, ia, ip0, q0, q1);
        if (threadIdx.x == 0) s_chunk = next;
    }
}

// The same in FP64 (precision 64): xbar += t^gamma x on the FP64 state, one
// sequence per thread of each chunk.
__device__ void average_pass64(const DevPlayer &P, const DevGames &gm, const IterArgs &ia, int64_t S) {
    __shared__ int s_chunk64;
    const int64_t nch = (S + kAvgChunk - 1) / kAvgChunk;
    for (;;) {
        if (threadIdx.x == 0) s_chunk64 = atomicAdd(&P.qavg[0], 1);
        __syncthreads();
        const int64_t c = s_chunk64;
        __syncthreads();
        if (c >= nch) break;
        const int64_t q1 = min((int64_t)S, (c + 1) * kAvgChunk);
        for (int64_t s = c * kAvgChunk + threadIdx.x; s < q1; s += blockDim.x) {
            const ItemParams64 pp = gm.par64[(int64_t)P.seq_game[s] * (kParamSpan + 1) + ia.pslot];
            const double xv = P.x64[s];
            if (pp.active && xv != 0.0) P.xbar64[s] += pp.w * xv;
        }
    }
}

// Shared state of the bottom-up and top-down loops of a CTA.
struct UpSmem {
    uint64_t bar[2];    // a buffer's own arrays
    SLvl lv[2][kMaxStagedLevels];
    UpTab tab[2][kMaxStagedLevels];
    ChildEv cev[2];
    ItemParams ip[2];
    UpPre pre;          // the unit to be issued next
    int4 win0[kPreWin]; // the first unit's x windows (copied once the previous kernel is done)
    int nwin0, win0_at; // their number and first record
    BulkCmd cmd[kUpArrays * kMaxStagedLevels];   // the producer's staged copies
    int unit[2];        // queue position of the unit in each buffer (n: none)
    int4 hq[2][2];      // its queue entry (header, tree record), for the consumers
    int armed[2];       // times each buffer's barrier was armed (bulk copies issued)
    int err;
};
struct DownSmem {
    uint64_t bar[2];
    SLvl lv[2][kMaxStagedLevels];
    DownTab tab[2][kMaxStagedLevels];
    BulkCmd cmd[kDownArrays * kMaxStagedLevels];   // the producer's staged copies
    ItemParams ip[2];
    int armed[2];       // times each buffer's barrier was armed (bulk copies issued)
    int cur, nxt, err, epoch;
};

// Before a CTA leaves a pass loop (normally or after a bounded wait gave up),
// thread 0 waits, bounded, for the last armed phase of each buffer's barrier:
// no bulk copy into this CTA's shared memory is then still in flight.
__device__ __forceinline__ void drain_copies(uint64_t *bar, const int *armed, int32_t *err) {
    if (threadIdx.x == 0)
        for (int b = 0; b < 2; b++)
            if (armed[b] > 0) mbar_wait(&bar[b], (uint32_t)(armed[b] - 1) & 1u, err);
}

// Up pass of one player (Alg. 2 ObserveUtility with the variant post-op of
// Alg. 3-5, and NextStrategy's regret matching).  Persistent CTAs take units
// from the bottom-up queue: every leaf, then the internal units deepest first.
// Warp 0 is the producer: while warps 1.. compute the current unit out of
// shared memory, it fetches the next unit, loads its parameters and starts its
// bulk copies into the other buffer.  An internal unit's own arrays are
// staged at once; its children's ev is copied in when its completion count
// shows all children done (a bounded wait: the children come earlier in the
// queue, every CTA works its units in queue order, and a child never waits
// for a later unit; a child at a static position of a CTA that is not yet
// resident is done once that CTA runs).  When `root_flag` is nonzero, the
// game's root unit sets the game's root_done word to it once every b of the
// game is final.
// Returns true when the CTA left the queues early: with a single game, it
// ended on the root with no unit after it, and registered its exit
// (launch_exit2) as it took the root, so that the launch's last exit (and,
// for a separate top-down launch, the kernel's end) does not wait for the
// root's exit path; such a CTA also skips the average pass, which the
// others complete.  With several games every CTA may end on a root, so none
// leaves early.
__device__ bool up_loop(const DevPlayer &P, const DevGames &gm, const float *__restrict__ xo, const IterArgs &ia,
                        unsigned char *const *bufs, UpSmem &S, int root_flag) {
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n = P.n_up;
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
        // a context whose earlier wait gave up does no more work (its
        // results are void): the remaining launches of a graph finish at once
        S.err = __ldcg(P.err) != 0;
        S.armed[0] = S.armed[1] = 0;
    }
    __syncthreads();
    if (S.err) return false;
    uint32_t ph[2] = {0u, 0u};
    int buf = 0;
    // The producer keeps a pipeline a round deep: the unit in each buffer
    // (S.unit), the unit to be issued next with everything its issue reads
    // (S.pre), and the queue position after that (pend, lane 0), whose
    // fetch was started a round earlier.  Every position comes from the
    // queue counter, so only a running CTA ever holds a unit (a unit that
    // another CTA waits for is never held by a CTA that is not yet resident);
    // a CTA claims its second position only once its first is issued, so
    // that the CTAs running at the start each hold one unit before any holds
    // two.  Positions only grow along a CTA's pipeline.
    auto fetch = [&]() { return atomicAdd(&P.qup[0], 1); };
    int pend = n;
    int4 h0 = make_int4(0, 0, 0, 0), q0 = h0;
    // prologue, overlapping the previous kernel: nothing read here is written
    // by it (the other player's x waits)
    if (warp == 0) {
        int p0 = n, p1 = n;
        if (tid == 0) p0 = fetch();
        p0 = __shfl_sync(0xffffffffu, p0, 0);
        if (p0 < n) {
            h0 = P.upq[2 * p0];
            q0 = P.upq[2 * p0 + 1];
            up_prefetch(P, gm, ia, p0, h0, q0, S.pre);
            cp_async_wait_all();
            __syncwarp();
            if (tid == 0) S.ip[0] = S.pre.ip;
            if (h0.w & kStaged) {
                issue_up(P, xo, S.pre, bufs[0], &S.bar[0], S.lv[0], S.tab[0], &S.cev[0], S.cmd, true);
                if (tid == 0) S.armed[0]++;
            }
            for (int w = tid; w < min(unit_nwin(h0), kPreWin); w += 32) S.win0[w] = S.pre.win[w];
        }
        if (tid == 0) {
            S.nwin0 = (p0 < n && (h0.w & kStaged)) ? unit_nwin(h0) : 0;
            S.win0_at = q0.w;
        }
        if (tid == 0) {
            S.unit[0] = p0 < n ? p0 : n;
            S.hq[0][0] = h0;
            S.hq[0][1] = q0;
        }
        if (tid == 0 && p0 < n) p1 = fetch();
        p1 = __shfl_sync(0xffffffffu, p1, 0);
        if (tid == 0) pend = p1 < n ? fetch() : n;
        if (p1 < n) up_prefetch(P, gm, ia, p1, P.upq[2 * p1], P.upq[2 * p1 + 1], S.pre);
        else if (tid == 0) S.pre.pos = n;
    }
    __syncthreads();
    // wait before letting the next kernel start: then at most two kernels of
    // the stream are resident, and a launch never shares its queue words with
    // a running one
    pdl_wait();
    pdl_trigger();
    // the first unit's x windows (the other player's x is final now), by
    // every thread; more windows than were kept come from global memory
    {
        const int nw = S.nwin0;
        if (nw > 0) {
            copy_up_x(xo, nw, nw <= kPreWin ? S.win0 : P.win + S.win0_at, S.tab[0], tid, blockDim.x);
            cp_async_wait_all();
        }
        __syncthreads();
    }
    int done_par = -1;   // parent of the previous unit, counted by the producer
    int cur = S.unit[0];
    bool early = false;
    while (cur < n) {
        // the unit's queue entry, as the producer kept it
        const int4 h = S.hq[buf][0];
        const int4 q = S.hq[buf][1];
        const int u = q.x;
        const int2 tr = make_int2(q.y, q.z);
        const bool staged = (h.w & kStaged) != 0, internal = tr.y > 0, root = tr.x < 0;
        if (staged) {
            if (warp != 0 && !mbar_wait(&S.bar[buf], ph[buf], P.err)) S.err = 1;
            ph[buf] ^= 1u;
        }
        __syncthreads();
        if (S.err) break;
        if (root && S.pre.pos >= n && !early && gridDim.x > 1 && P.G == 1) {   // another CTA does the average pass
            launch_exit2(P.qup, P.qavg);
            early = true;
        }
        const ItemParams ip = S.ip[buf];
        if (warp == 0) {
            // producer: issue the prefetched unit into the other buffer;
            // count the previous unit at its parent (its results were
            // written before the barrier above); then prefetch the unit after
            // the next one, whose queue position came last round, and start
            // fetching the next position
            // the queue entry of the unit after next (its position came
            // last round): loaded now, used after the issue below
            const int p = __shfl_sync(0xffffffffu, pend, 0);
            int4 hp = make_int4(0, 0, 0, 0), qp = hp;
            if (p < n) {
                hp = P.upq[2 * p];
                qp = P.upq[2 * p + 1];
            }
            // the next unit, whose records were copied in last round
            cp_async_wait_all();
            __syncwarp();
            const int nx = S.pre.pos;
            if (nx < n) {
                if (tid == 0) S.ip[buf ^ 1] = S.pre.ip;
                if (S.pre.h.w & kStaged) {
                    issue_up(P, xo, S.pre, bufs[buf ^ 1], &S.bar[buf ^ 1], S.lv[buf ^ 1], S.tab[buf ^ 1],
                             &S.cev[buf ^ 1], S.cmd, false);
                    if (tid == 0) S.armed[buf ^ 1]++;
                }
            }
            if (tid == 0) {
                S.unit[buf ^ 1] = nx;
                S.hq[buf ^ 1][0] = S.pre.h;
                S.hq[buf ^ 1][1] = S.pre.q;
            }
            if (tid == 0 && done_par >= 0) {
                __threadfence();
                atomicAdd(&P.unit_cnt[done_par], 1);
            }
            __syncwarp();   // S.pre is read: the next one may overwrite it
            if (tid == 0) pend = p < n ? fetch() : n;
            if (p < n) up_prefetch(P, gm, ia, p, hp, qp, S.pre);
            else if (tid == 0) S.pre.pos = n;
        } else if (ip.active) {
            if (internal) {
                // all children done, then their ev, copied by every consumer
                // thread (the acquire above orders it through the barrier)
                if (tid == 32) {
                    if (!flag_wait(&P.unit_cnt[u], tr.y, P.err, P.wait_ns)) S.err = 1;
                    P.unit_cnt[u] = 0;
                }
                consumer_sync();
                if (staged && !S.err) {
                    copy_child_ev(S.cev[buf], tid - kProducerThreads, (int)blockDim.x - kProducerThreads);
                    cp_async_wait_all();
                }
                consumer_sync();
            }
            if (staged && !S.err) {
                up_gather(xo, h.y, S.lv[buf], S.tab[buf], internal);
                compute_up(P, ia, ip, h.y, S.lv[buf], S.tab[buf], &S.cev[buf], internal);
                if (internal && !root && tid == 32) {
                    // the parent reads only this unit's top-level ev, stored
                    // (with r and b) by the steps before the last consumer
                    // barrier: count the unit there now
                    __threadfence();
                    atomicAdd(&P.unit_cnt[tr.x], 1);
                }
            }
        }
        __syncthreads();
        if (S.err) break;
        if (ip.active) {
            if (!staged) run_up<MODE_CFR>(P, xo, ia, ip, h.y, P.ranges + h.z, bufs[buf]);
            if (tid == 0 && root && ia.first_of_iter) gm.t_done[h.x] = ip.t;
        }
        if (tid == 0 && root && root_flag) {
            // the game's bottom-up pass is complete: every b final (set for
            // games masked off too, whose top-down units then do nothing)
            __threadfence();
            st_release(&P.root_done[h.x], root_flag);
        }
        // the producer counts the unit at its parent at the start of the next
        // round (a staged internal unit has counted itself already)
        done_par = (ip.active && !(staged && internal)) ? tr.x : -1;
        cur = S.unit[buf ^ 1];
        buf ^= 1;
    }
    // the last unit's count (nothing else of this CTA is pending; records
    // prefetched for a unit not taken after an error land first, and so do
    // bulk copies into a buffer whose unit was not computed)
    cp_async_wait_all();
    __syncthreads();
    drain_copies(S.bar, S.armed, P.err);
    if (tid == 0 && done_par >= 0) {
        __threadfence();
        atomicAdd(&P.unit_cnt[done_par], 1);
    }
    __syncthreads();
    return early;
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_up_staged(DevPlayer P, DevGames gm, const float *__restrict__ xo, IterArgs ia, int item_bytes) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *bufs[2] = {smem, smem + item_bytes};
    __shared__ UpSmem S;
    if (!up_loop(P, gm, xo, ia, bufs, S, 0)) {
        if (ia.average && !S.err) average_pass(P, gm, ia, P.S);
        __syncthreads();
        launch_exit2(P.qup, P.qavg);
    }
}

// one unit top-down from global memory (units too large to stage): its
// ancestor chain (the first n_anc levels, from the game's root) into its own
// scratch area xa, then its own levels into x
__device__ void run_down(const DevPlayer &P, int nlvl, int n_anc, const int32_t *rng, float *xa) {
    int aoff = 0, poff = 0;   // scratch offset of this level / of the level above
    for (int k = 0; k < nlvl; k++) {
        const int s0 = rng[kLvl * k + 2];
        const int ps0 = k > 0 ? rng[kLvl * (k - 1) + 2] : 0;
        // parents: the level above, in the scratch area while it is an ancestor level
        const bool par_anc = k > 0 && k - 1 < n_anc, anc = k < n_anc;
        for (int j = rng[kLvl * k] + (int)threadIdx.x; j < rng[kLvl * k + 1]; j += blockDim.x) {
            const int par = P.inf_par[j];
            const float xp = par < 0 ? 1.f : par_anc ? __ldcg(&xa[poff + (par - ps0)]) : __ldcg(&P.x[par]);
            for (int s = P.inf_seq[j]; s < P.inf_seq[j + 1]; s++) {
                const float v = xp * P.b[s];
                if (anc) xa[aoff + (s - s0)] = v;
                else P.x[s] = v;
            }
        }
        __syncthreads();
        if (anc) {
            poff = aoff;
            aoff += rng[kLvl * k + 3] - s0;
        }
    }
}


// the same in FP64 (precision 64); every unit keeps its ancestors' x in its
// own scratch area
__device__ void run_down64(const DevPlayer &P, int nlvl, int n_anc, const int32_t *rng, double *xa) {
    int aoff = 0, poff = 0;
    for (int k = 0; k < nlvl; k++) {
        const int s0 = rng[kLvl * k + 2];
        const int ps0 = k > 0 ? rng[kLvl * (k - 1) + 2] : 0;
        const bool par_anc = k > 0 && k - 1 < n_anc, anc = k < n_anc;
        for (int j = rng[kLvl * k] + (int)threadIdx.x; j < rng[kLvl * k + 1]; j += blockDim.x) {
            const int par = P.inf_par[j];
            const double xp = par < 0 ? 1.0 : par_anc ? __ldcg(&xa[poff + (par - ps0)]) : __ldcg(&P.x64[par]);
            for (int s = P.inf_seq[j]; s < P.inf_seq[j + 1]; s++) {
                const double v = xp * P.b64[s];
                if (anc) xa[aoff + (s - s0)] = v;
                else P.x64[s] = v;
            }
        }
        __syncthreads();
        if (anc) {
            poff = aoff;
            aoff += rng[kLvl * k + 3] - s0;
        }
    }
}

// Top-down pass of an FP64 iteration: every top-down unit from the queue,
// worked from global memory.
__global__ void __launch_bounds__(kThreads) k_down64(DevPlayer P, DevGames gm, IterArgs ia) {
    __shared__ int s_item, s_err;
    if (threadIdx.x == 0) s_err = __ldcg(P.err) != 0;
    __syncthreads();
    for (;;) {
        if (s_err) break;
        if (threadIdx.x == 0) s_item = atomicAdd(&P.qdn[0], 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= P.n_units) break;
        const int4 h = P.downq[2 * it];
        const int4 q = P.downq[2 * it + 1];
        if (!gm.par64[(int64_t)h.x * (kParamSpan + 1) + ia.pslot].active) continue;
        run_down64(P, h.y, h.w >> kAncShift, P.ranges + h.z, P.xanc64 + q.w);
    }
    launch_exit(P.qdn);
}

// Down pass (Alg. 2 NextStrategy: y += L^T y, x = A^T y; the average
// xbar += t^gamma x was done by the bottom-up pass's CTAs before).  Every
// unit recomputes the next x of its ancestor chain (the infosets above its
// top level, up to the game's root) from the final b, so the units are
// independent of one another.  With `wait_roots` (the loop follows
// this player's bottom-up loop in the same launch) a unit's b is copied in,
// and the unit computed, only once its game's root_done word shows the
// bottom-up pass of that game complete (a bounded wait; the root unit was
// taken by a running CTA before any top-down unit was).
// Returns true when the CTA registered its exit (launch_exit) as it took its
// last unit, as the bottom-up loop does.
__device__ bool down_loop(const DevPlayer &P, const DevGames &gm, const IterArgs &ia, unsigned char *const *bufs,
                          DownSmem &S, bool wait_roots, int avg_flag = 0) {
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n = P.n_units;
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
        S.err = __ldcg(P.err) != 0;   // see up_loop
        S.cur = S.err ? n : atomicAdd(&P.qdn[0], 1);
        S.armed[0] = S.armed[1] = 0;
    }
    __syncthreads();
    const int flag = S.epoch + 1;
    uint32_t ph[2] = {0u, 0u};
    int cur = S.cur, buf = 0;
    // warp 0: the game's bottom-up pass must be complete before b is read;
    // every lane then acquires the flag itself, since every lane issues copies
    bool avg_seen = avg_flag == 0;
    auto root_ready = [&](int g) {
        if (!wait_roots) return true;
        bool ok = true;
        if ((tid & 31) == 0 && !avg_seen) ok = avg_seen = flag_wait(&P.qavg[2], avg_flag, P.err, P.wait_ns);
        if ((tid & 31) == 0 && ok) ok = flag_wait(&P.root_done[g], flag, P.err, P.wait_ns);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) ok = ld_acquire(&P.root_done[g]) == flag;
        return __all_sync(0xffffffffu, ok) != 0;
    };
    // prologue, overlapping the previous kernel (or this launch's bottom-up
    // loop): the first unit's index arrays, by the producer's bulk copies;
    // then, once that kernel is done, its b and parents' x, copied by every
    // thread at once (16-byte cp.async through L2)
    const int4 h0 = cur < n ? P.downq[2 * cur] : make_int4(0, 0, 0, 0);
    const bool st0 = cur < n && (h0.w & kStaged);
    if (warp == 0) {
        if (st0) {
            issue_down(P, h0, bufs[0], &S.bar[0], S.lv[0], S.tab[0], S.cmd, kDownOwn | kDownArm, 0);
            if (tid == 0) S.armed[0]++;
        }
        // the parameter table is written ahead of the passes, never by the
        // kernel this one may overlap
        if (tid == 0 && cur < n) S.ip[0] = unit_params(gm, ia, h0.x);
        pdl_wait();
        // With no more units than CTAs every unit is some CTA's first, and a
        // second claim could only move units onto CTAs that already hold one
        // (those that started first), leaving others idle: the pass is one
        // round.  Otherwise the second position is claimed only now, once
        // every CTA that was resident while the previous kernel ran holds
        // its first.
        if (tid == 0) S.nxt = (cur < n && n > (int)gridDim.x) ? atomicAdd(&P.qdn[0], 1) : n;
        if (cur < n && !root_ready(h0.x) && tid == 0) S.err = 1;
    }
    __syncthreads();
    pdl_trigger();
    pdl_wait();
    if (st0 && !S.err) {
        for (int k = 0; k < h0.y; k++) {
            const BulkCmd c = S.cmd[kDownArrays * k];   // b
            for (uint32_t o = 16u * tid; o < c.bytes; o += 16u * blockDim.x)
                cp_async16_cg_to(c.dst + o, (const unsigned char *)c.src + o);
        }
        cp_async_wait_all();
    }
    __syncthreads();
    int nxt = S.nxt;
    bool early = false;
    while (cur < n && !S.err) {
        const int4 h = P.downq[2 * cur];
        const bool staged = (h.w & kStaged) != 0;
        if (nxt >= n && !early) {   // the last unit of this CTA: no more queue use
            launch_exit(P.qdn);
            early = true;
        }
        if (staged) {
            if (warp != 0 && !mbar_wait(&S.bar[buf], ph[buf], P.err)) S.err = 1;
            ph[buf] ^= 1u;
        }
        __syncthreads();
        if (S.err) break;
        const ItemParams ip = S.ip[buf];
        if (warp == 0) {
            if (nxt < n) {
                const int4 hn = P.downq[2 * nxt];
                if (!root_ready(hn.x) && tid == 0) S.err = 1;
                if (hn.w & kStaged) {
                    issue_down(P, hn, bufs[buf ^ 1], &S.bar[buf ^ 1], S.lv[buf ^ 1], S.tab[buf ^ 1], S.cmd,
                               kDownOwn | kDownB | kDownArm, 0);
                    if (tid == 0) S.armed[buf ^ 1]++;
                }
                if (tid == 0) S.ip[buf ^ 1] = unit_params(gm, ia, hn.x);
            }
            if (tid == 0) S.nxt = nxt < n ? atomicAdd(&P.qdn[0], 1) : n;
        } else if (ip.active && staged) {
            compute_down(P, h.y, h.w >> kAncShift, S.lv[buf], S.tab[buf]);
        }
        __syncthreads();
        const int nxt2 = S.nxt;
        if (ip.active && !staged)
            run_down(P, h.y, h.w >> kAncShift, P.ranges + h.z, P.xanc + P.downq[2 * cur + 1].w);
        cur = nxt;
        nxt = nxt2;
        buf ^= 1;
    }
    cp_async_wait_all();
    drain_copies(S.bar, S.armed, P.err);
    __syncthreads();
    return early;
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_down_staged(DevPlayer P, DevGames gm, IterArgs ia, int item_bytes) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *bufs[2] = {smem, smem + item_bytes};
    __shared__ DownSmem S;
    if (threadIdx.x == 0) S.epoch = 0;
    if (!down_loop(P, gm, ia, bufs, S, false)) launch_exit(P.qdn);
}

// One player's whole half-step in one launch (alternating updates): the
// bottom-up loop, then, as each CTA runs out of bottom-up units, the top-down
// loop; a game's top-down units start once that game's root unit is done.
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_half_step(DevPlayer P, DevGames gm, const float *__restrict__ xo, IterArgs up_ia, IterArgs dn_ia,
                int item_bytes) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *bufs[2] = {smem, smem + item_bytes};
    __shared__ UpSmem SU;
    __shared__ DownSmem SD;
    // this launch's root flag is the top-down epoch + 1: the previous launch
    // on these queue words finished before this one started (each pass lets
    // the next kernel start only after its own wait on the previous one)
    // likewise the average pass's: the top-down loop overwrites x only once
    // every CTA has left the average pass
    __shared__ int s_avg;
    if (threadIdx.x == 0) {
        SD.epoch = __ldcg(&P.qdn[2]);
        s_avg = __ldcg(&P.qavg[2]) + 1;
    }
    __syncthreads();
    if (!up_loop(P, gm, xo, up_ia, bufs, SU, SD.epoch + 1)) {
        if (up_ia.average && !SU.err) average_pass(P, gm, up_ia, P.S);
        __syncthreads();
        launch_exit2(P.qup, P.qavg);
    }
    __syncthreads();
    if (!SU.err) {
        if (!down_loop(P, gm, dn_ia, bufs, SD, true, up_ia.average ? s_avg : 0)) launch_exit(P.qdn);
    } else {
        launch_exit(P.qdn);
    }
}

// uniform behavioural strategy (regret matching of r = 0)
__global__ void k_uniform(DevPlayer P, int64_t J) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J; j += (int64_t)gridDim.x * blockDim.x) {
        const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
        const float v = __frcp_rn((float)(s1 - s0));
        for (int s = s0; s < s1; s++) P.b[s] = v;
        if (P.fp64)
            for (int s = s0; s < s1; s++) P.b64[s] = 1.0 / (double)(s1 - s0);
    }
}

// the state of sequence s as FP64, from whichever precision the context keeps
__device__ __forceinline__ double st_xbar(const DevPlayer &P, int64_t s) {
    if (P.fp64) return P.xbar64[s];
    const float2 v = P.xbar[s];
    return (double)v.x + (double)v.y;
}
__device__ __forceinline__ double st_r(const DevPlayer &P, int64_t s) {
    if (P.fp64) return P.r64[s];
    const float2 v = P.r[s];
    return (double)v.x + (double)v.y;
}
__device__ __forceinline__ double st_b(const DevPlayer &P, int64_t s) { return P.fp64 ? P.b64[s] : (double)P.b[s]; }
__device__ __forceinline__ double st_x(const DevPlayer &P, int64_t s) { return P.fp64 ? P.x64[s] : (double)P.x[s]; }

// normalised average (FP64) for the best-response pass; current x where no
// iteration has been averaged yet
__global__ void k_normalize(DevPlayer P, int64_t S) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const int g = P.seq_game[s];
        const double den = st_xbar(P, g);
        P.xnorm[s] = den > 0.0 ? st_xbar(P, s) / den : st_x(P, s);
    }
}

// state of one game in caller order (FP64): r, b, xbar (empty first)
__global__ void k_get_state(DevPlayer P, const int32_t *ext_inf, const int32_t *ext_seq0, int g, int Jg,
                            double *out_r, double *out_b, double *out_xbar) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) out_xbar[0] = st_xbar(P, g);
    if (k >= Jg) return;
    const int j = ext_inf[k];
    const int base = ext_seq0[k];
    const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
    for (int s = s0; s < s1; s++) {
        const int o = base + (s - s0);
        out_r[o] = st_r(P, s);
        out_b[o] = st_b(P, s);
        out_xbar[1 + o] = st_xbar(P, s);
    }
}

__global__ void k_set_state(DevPlayer P, const int32_t *ext_inf, const int32_t *ext_seq0, int g, int Jg,
                            const double *in_r, const double *in_b, const double *in_xbar) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        if (P.fp64) P.xbar64[g] = in_xbar[0];
        else P.xbar[g] = ff_from_double(in_xbar[0]);
    }
    if (k >= Jg) return;
    const int j = ext_inf[k];
    const int base = ext_seq0[k];
    const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
    for (int s = s0; s < s1; s++) {
        const int o = base + (s - s0);
        if (P.fp64) {
            P.r64[s] = in_r[o];
            P.b64[s] = in_b[o];
            P.xbar64[s] = in_xbar[1 + o];
        } else {
            P.r[s] = ff_from_double(in_r[o]);
            P.b[s] = (float)in_b[o];
            P.xbar[s] = ff_from_double(in_xbar[1 + o]);
        }
    }
}

// average behavioural strategy of one game: xbar[(j,a)] / xbar[p_j] (FP64)
__global__ void k_average(DevPlayer P, const int32_t *ext_inf, const int32_t *ext_seq0, int Jg, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Jg) return;
    const int j = ext_inf[k];
    const int base = ext_seq0[k];
    const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
    const double den = st_xbar(P, P.inf_par[j]);
    for (int s = s0; s < s1; s++) out[base + (s - s0)] = den > 0.0 ? st_xbar(P, s) / den : 1.0 / (double)(s1 - s0);
}

__global__ void k_set_t(int32_t *t_done, int g, int32_t t) { t_done[g] = t; }

// One game's state (r, b, xbar, in either precision) from another context
// holding the same game, infoset by infoset in caller order; x is rebuilt
// afterwards.
__global__ void k_copy_game(DevPlayer D, const int32_t *dext, int gd, DevPlayer S, const int32_t *sext, int gs, int Jg) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        if (D.fp64) D.xbar64[gd] = S.xbar64[gs];
        else D.xbar[gd] = S.xbar[gs];
    }
    if (k >= Jg) return;
    const int jd = dext[k], js = sext[k];
    const int d0 = D.inf_seq[jd], s0 = S.inf_seq[js], na = S.inf_seq[js + 1] - s0;
    for (int a = 0; a < na; a++) {
        if (D.fp64) {
            D.r64[d0 + a] = S.r64[s0 + a];
            D.b64[d0 + a] = S.b64[s0 + a];
            D.xbar64[d0 + a] = S.xbar64[s0 + a];
        } else {
            D.r[d0 + a] = S.r[s0 + a];
            D.b[d0 + a] = S.b[s0 + a];
            D.xbar[d0 + a] = S.xbar[s0 + a];
        }
    }
}
__global__ void k_copy_t(int32_t *dt, int gd, const int32_t *st, int gs) { dt[gd] = st[gs]; }

// current sequence-form strategy (empty sequence first) and per-infoset ev of
// one game in caller order (FP64)
__global__ void k_get_values(DevPlayer P, const int32_t *ext_inf, const int32_t *ext_seq0, int g, int Jg,
                             double *out_x, double *out_ev) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) out_x[0] = st_x(P, g);
    if (k >= Jg) return;
    const int j = ext_inf[k];
    const int base = ext_seq0[k];
    out_ev[k] = P.fp64 ? P.evc64[j] : (double)P.ev[j];
    const int s0 = P.inf_seq[j], s1 = P.inf_seq[j + 1];
    for (int s = s0; s < s1; s++) out_x[1 + base + (s - s0)] = st_x(P, s);
}

}  // namespace cfrb

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
namespace {

thread_local std::string g_last_error;
thread_local const char *g_last_error_static = nullptr;

int set_err(int code, const std::string &m) {
    g_last_error = m;
    g_last_error_static = nullptr;
    return code;
}

// error with a static message: no allocation on this path
int set_err_static(int code, const char *m) {
    g_last_error_static = m;
    return code;
}

// Launch shapes of the staged passes: threads per CTA, CTAs per SM and the
// unit buffer (two per CTA).  More, smaller CTAs per SM overlap one CTA's
// barrier waits and copy latency with another's compute.
using UpFn = void (*)(DevPlayer, DevGames, const float *, IterArgs, int);
using DownFn = void (*)(DevPlayer, DevGames, IterArgs, int);
using HalfFn = void (*)(DevPlayer, DevGames, const float *, IterArgs, IterArgs, int);
struct StagedConfig {
    int threads, ctas_per_sm, item_bytes;
    UpFn up;
    DownFn down;
    HalfFn half;
};
#define CFR_SHAPE(nt, minb, kb) {nt, minb, kb * 1024, k_up_staged<nt, minb>, k_down_staged<nt, minb>, k_half_step<nt, minb>}
const StagedConfig kConfigs[] = {
    CFR_SHAPE(512, 1, 96), CFR_SHAPE(256, 2, 48), CFR_SHAPE(256, 3, 32), CFR_SHAPE(512, 2, 48), CFR_SHAPE(256, 4, 24),
    CFR_SHAPE(384, 2, 48), CFR_SHAPE(320, 2, 48),
};
#undef CFR_SHAPE
constexpr int kNumConfigs = (int)(sizeof(kConfigs) / sizeof(kConfigs[0]));
constexpr int kDefaultConfig = 6;   // 320 threads, 2 CTAs per SM, 48 KB buffers
constexpr int kManyConfig = 2;      // 256 threads, 3 CTAs per SM, 32 KB buffers
constexpr int64_t kLargeGameNodes = 1000000;
// The launch shape used when none is chosen: a single game of at least 1M
// nodes runs fastest with 48 KB units on two CTAs per SM (fewer unit tiers);
// smaller games and batches with 32 KB units on three (more units at once):
// measured 10-12% faster on batches of 10^3-10^6-node games, within 1% on
// one large game.
int pick_config(int64_t n_games, int64_t total_nodes) {
    return (n_games == 1 && total_nodes >= kLargeGameNodes) ? kDefaultConfig : kManyConfig;
}


struct PlayerBuf {
    DevPlayer d{};
    int32_t *ext_inf = nullptr, *ext_seq0 = nullptr;
    int64_t S = 0, J = 0, n_units = 0, n_up = 0;
    int n_levels = 0;
    int grid_up = 1, grid_up_br = 1, grid_down = 1, grid_half = 1, grid_up64 = 1, grid_down64 = 1;
    size_t smem_br = 0;
    std::vector<int32_t> game_J, game_S;
    std::vector<int64_t> game_jbase;
};

struct GraphKey {
    int variant, mode, k;
    double a, b, g;
    bool operator<(const GraphKey &o) const {
        return std::tie(variant, mode, k, a, b, g) < std::tie(o.variant, o.mode, o.k, o.a, o.b, o.g);
    }
};

}  // namespace

struct cfr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t G = 0, Z = 0;
    PlayerBuf pl[2];
    int32_t *t_done = nullptr;
    uint8_t *active = nullptr;
    uint8_t *active_keep = nullptr; // device copy of the caller's mask, restored after a
                                    // best-response pass (which runs every game)
    ItemParams *par = nullptr;      // per-game parameter table (kParamSpan + 1 entries)
    ItemParams64 *par64 = nullptr;  // the same in FP64 (precision 64 only)
    bool fp64 = false;              // precision 64: the iteration runs in FP64 from global memory
    int32_t *pbase = nullptr;
    int32_t *mixed = nullptr;   // set by k_params when the games' parameters differ
    double *br[2] = {nullptr, nullptr};
    double *scratch = nullptr;   // FP64 transfer area: 3 * (max S + 1)
    int64_t scratch_n = 0;
    int update_mode = CFR_UPDATES_DEFAULT;
    int graph_k = 64;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::vector<void *> allocs;
    std::vector<int64_t> game_nodes, game_nnz;
    std::vector<uint8_t> active_host;
    int64_t dev_bytes = 0, h2d_bytes = 0;
    int cfg = kDefaultConfig;       // staged launch shape (kConfigs)
    bool pdl = true;                // passes may overlap the previous pass's tail (not while profiling)
    bool split = false;             // alternating schedule: separate bottom-up and top-down launches
    int threads = 256;              // threads of a staged CTA
    int item_bytes = 48 * 1024;     // one staged unit buffer (two per CTA)
    size_t smem_staged = 0;
    int32_t *err = nullptr;         // device error word (bounded waits)
    bool poisoned = false;
    bool values = false;            // up passes store every infoset's ev (cfr_get_values)
    uint64_t wait_ns = kFlagWaitNs; // longest wait of a unit for the units it depends on
    int64_t launches = 0;           // kernels launched so far (graph replays count their kernels)
    std::map<GraphKey, int64_t> graph_kernels;   // kernels in each captured graph
};

namespace {

#define CU(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return set_err(e_ == cudaErrorMemoryAllocation ? CFR_ERR_OOM : CFR_ERR_CUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_));          \
    } while (0)

#define TRY(x)               \
    do {                     \
        int rc_ = (x);       \
        if (rc_) return rc_; \
    } while (0)

// Every entry point that does CUDA set-up work or waits for the device --
// loading (allocations, uploads, first kernels), iterating (graph capture and
// instantiation), reading or writing state through host memory, exploitability,
// synchronising, freeing -- runs under one process-wide lock.  A graph capture
// in one thread then never overlaps another thread's allocation, free,
// pageable copy or kernel-module load through this library, any of which can
// invalidate the capture (contexts loaded on worker threads while another
// thread iterates).  The host compile of a load runs outside the lock.
std::recursive_mutex &setup_mutex() {
    static std::recursive_mutex m;
    return m;
}

template <class T>
int dalloc(cfr_ctx *c, T **p, size_t n) {
    void *q = nullptr;
    // 32 bytes of tail padding: staged copies round their ranges out to 16 bytes
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T) + 32;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(CFR_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    c->dev_bytes += (int64_t)bytes;
    *p = (T *)q;
    return CFR_OK;
}

template <class T>
int upload(cfr_ctx *c, T **p, const std::vector<T> &v) {
    TRY(dalloc(c, p, v.size()));
    if (!v.empty()) CU(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    c->h2d_bytes += (int64_t)(v.size() * sizeof(T));
    return CFR_OK;
}

DevGames dev_games(const cfr_ctx *c) {
    return DevGames{c->t_done, c->active, nullptr, c->par, c->pbase, c->mixed, c->par64};
}

// the parameter table for the next kParamSpan iterations of every game
int launch_params(cfr_ctx *c, int variant, double alpha, double beta, double gamma) {
    IterArgs ia{variant, 0, 0.f, alpha, beta, gamma, 0, 0, 0};
    const int64_t n = c->G * (kParamSpan + 1);
    CU(cudaMemsetAsync(c->mixed, 0, sizeof(int32_t), c->stream));
    k_params<<<(unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 4096), kThreads, 0, c->stream>>>(
        dev_games(c), ia, (int)c->G);
    CU(cudaGetLastError());
    return CFR_OK;
}

// x of player p from the current b (top-down, no averaging), for every game
// whatever the active mask
int launch_rebuild_x(cfr_ctx *c, int p) {
    PlayerBuf &B = c->pl[p];
    const bool masked = std::find(c->active_host.begin(), c->active_host.end(), 0) != c->active_host.end();
    if (masked) CU(cudaMemsetAsync(c->active, 1, c->G, c->stream));
    TRY(launch_params(c, 0, 0.0, 0.0, 0.0));
    IterArgs ia{};
    ia.average = 0;
    if (c->fp64)
        k_down64<<<B.grid_down64, kThreads, 0, c->stream>>>(B.d, dev_games(c), ia);
    else
        kConfigs[c->cfg].down<<<B.grid_down, c->threads, c->smem_staged, c->stream>>>(B.d, dev_games(c), ia,
                                                                                       c->item_bytes);
    CU(cudaGetLastError());
    if (masked) CU(cudaMemcpyAsync(c->active, c->active_keep, c->G, cudaMemcpyDeviceToDevice, c->stream));
    return CFR_OK;
}

// Launch a pass kernel; with pdl it may start while the previous kernel on the
// stream finishes (programmatic dependent launch: the kernel waits for that
// kernel itself before it reads anything the kernel writes).
template <class... P, class... A>
cudaError_t launch_pass(void (*fn)(P...), int grid, int threads, size_t smem, cudaStream_t st, bool pdl, A &&...a) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, fn, std::forward<A>(a)...);
}

// one iteration: NextStrategy/ObserveUtility for both players (Alg. 2), in the
// alternating or simultaneous schedule (Sec. 3.5.1).  Each pass may overlap
// the previous one's tail (not when timing the passes one by one, and not
// right after the parameter table is refilled).
int launch_iteration(cfr_ctx *c, int variant, double alpha, double beta, double gamma, bool alternating,
                     int k, int64_t *nlaunch, cudaEvent_t *ev = nullptr) {
    const bool params = (k % kParamSpan) == 0;
    const int pslot = k % kParamSpan + 1;
    if (params) TRY(launch_params(c, variant, alpha, beta, gamma));
    *nlaunch += params ? 1 : 0;
    const DevGames gm = dev_games(c);
    // every pass of the k-th iteration since the table was filled runs at
    // t = t_done + k + 1 of that moment
    const int keep = c->values ? 1 : 0;
    IterArgs up1{variant, 1, +1.f, alpha, beta, gamma, 1, pslot, keep};
    IterArgs up2{variant, 0, -1.f, alpha, beta, gamma, 1, pslot, keep};
    IterArgs dn{variant, 0, 0.f, alpha, beta, gamma, 1, pslot, keep};
    PlayerBuf &A = c->pl[0], &B = c->pl[1];
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], c->stream);
    };
    const size_t sm = c->smem_staged;
    const int ib = c->item_bytes, nt = c->threads;
    const UpFn up = kConfigs[c->cfg].up;
    const DownFn down = kConfigs[c->cfg].down;
    const bool pdl = (ev == nullptr) && c->pdl;
    const bool pdl0 = pdl && !params;
    const float *x1 = A.d.x, *x2 = B.d.x;
    mark(0);
    if (c->fp64) {
        // precision 64: the same schedule with the FP64 passes, from global memory
        const double *y1 = A.d.x64, *y2 = B.d.x64;
        auto up64 = [&](PlayerBuf &P, const double *xo, const IterArgs &ia) {
            k_up<MODE_CFR64><<<P.grid_up64, kThreads, P.smem_br, c->stream>>>(P.d, gm, (const void *)xo, ia);
        };
        auto down64 = [&](PlayerBuf &P) { k_down64<<<P.grid_down64, kThreads, 0, c->stream>>>(P.d, gm, dn); };
        if (alternating) {
            up64(A, y2, up1);
            mark(1);
            down64(A);
            mark(2);
            up64(B, y1, up2);
            mark(3);
            down64(B);
        } else {
            up64(A, y2, up1);
            mark(1);
            up64(B, y1, up2);
            mark(2);
            down64(A);
            mark(3);
            down64(B);
        }
        *nlaunch += 4;
        mark(4);
        CU(cudaGetLastError());
        return CFR_OK;
    }
    if (alternating && !c->split && !ev) {
        const HalfFn half = kConfigs[c->cfg].half;
        CU(launch_pass(half, A.grid_half, nt, sm, c->stream, pdl0, A.d, gm, x2, up1, dn, ib));
        CU(launch_pass(half, B.grid_half, nt, sm, c->stream, pdl, B.d, gm, x1, up2, dn, ib));
        *nlaunch += 2;
    } else if (alternating) {
        CU(launch_pass(up, A.grid_up, nt, sm, c->stream, pdl0, A.d, gm, x2, up1, ib));
        mark(1);
        CU(launch_pass(down, A.grid_down, nt, sm, c->stream, pdl, A.d, gm, dn, ib));
        mark(2);
        CU(launch_pass(up, B.grid_up, nt, sm, c->stream, pdl, B.d, gm, x1, up2, ib));
        mark(3);
        CU(launch_pass(down, B.grid_down, nt, sm, c->stream, pdl, B.d, gm, dn, ib));
        *nlaunch += 4;
    } else {
        CU(launch_pass(up, A.grid_up, nt, sm, c->stream, pdl0, A.d, gm, x2, up1, ib));
        mark(1);
        CU(launch_pass(up, B.grid_up, nt, sm, c->stream, pdl, B.d, gm, x1, up2, ib));
        mark(2);
        CU(launch_pass(down, A.grid_down, nt, sm, c->stream, pdl, A.d, gm, dn, ib));
        mark(3);
        CU(launch_pass(down, B.grid_down, nt, sm, c->stream, pdl, B.d, gm, dn, ib));
        *nlaunch += 4;
    }
    mark(4);
    CU(cudaGetLastError());
    return CFR_OK;
}

int occupancy_grid(const void *fn, int threads, size_t smem, int64_t n_work, int *grid) {
    int dev = 0, sms = 0, per = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem));
    if (per < 1) return set_err(CFR_ERR_CUDA, "kernel does not fit on an SM");
    const int64_t full = (int64_t)sms * per;
    *grid = (int)std::max<int64_t>(1, std::min<int64_t>(full, n_work));
    return CFR_OK;
}

int build_player(cfr_ctx *c, const Layout &L, int p) {
    const PlayerLayout &H = L.pl[p];
    PlayerBuf &B = c->pl[p];
    DevPlayer &d = B.d;
    B.S = H.S;
    B.J = H.J;
    B.n_units = (int64_t)H.dunits.size();
    B.n_up = (int64_t)H.up_queue.size();
    B.n_levels = H.n_levels;
    B.game_J = H.game_J;
    B.game_S = H.game_S;
    B.game_jbase = H.game_jbase;
    int32_t *p32;
    TRY(upload(c, &p32, H.inf_seq));
    d.inf_seq = p32;
    TRY(upload(c, &p32, H.seq_child));
    d.seq_child = p32;
    TRY(upload(c, &p32, H.inf_par));
    d.inf_par = p32;
    TRY(upload(c, &p32, H.seq_game));
    d.seq_game = p32;
    TRY(upload(c, &p32, H.m_ptr));
    d.m_ptr = p32;
    TRY(upload(c, &p32, H.m_col));
    d.m_col = p32;
    TRY(upload(c, &p32, H.lcol));
    d.lcol = p32;
    TRY(upload(c, &p32, H.rwin));
    d.rwin = (const int4 *)p32;
    TRY(upload(c, &p32, H.win));
    d.win = (const int4 *)p32;
    float *pf;
    TRY(upload(c, &pf, H.m_val));
    d.m_val = pf;
    double *pd;
    TRY(upload(c, &pd, H.m_val64));
    d.m_val64 = pd;
    std::vector<int4> units(H.units.size());
    std::vector<int2> tree(H.units.size());
    for (size_t k = 0; k < H.units.size(); k++) {
        const Unit &u = H.units[k];
        units[k] = make_int4(u.game, u.nlvl, u.rng, u.flags);
        tree[k] = make_int2(u.parent, u.nchild);
    }
    int4 *p4;
    TRY(upload(c, &p4, units));
    d.units = p4;
    int2 *p2;
    TRY(upload(c, &p2, tree));
    d.unit_tree = p2;
    TRY(upload(c, &p32, H.ranges));
    d.ranges = p32;
    // queue entries: {game, nlvl, rng, flags | x windows << 8}, {unit, parent,
    // child units, first x window}; a staged up unit's windows are one run
    auto queue = [&](const std::vector<int32_t> &qv, const std::vector<Unit> &units, bool up, const int4 **out) {
        std::vector<int4> q(2 * qv.size());
        for (size_t k = 0; k < qv.size(); k++) {
            const Unit &u = units[qv[k]];
            int32_t w0 = 0, nw = 0;
            if (up && (u.flags & kStaged)) {
                const int64_t rec = u.rng / kLvl;
                w0 = H.rwin[4 * rec];
                nw = H.rwin[4 * (rec + u.nlvl - 1) + 1] - w0;
            }
            if (!up) w0 = H.danc_off[qv[k]];   // top-down: the unit's ancestor scratch
            q[2 * k] = make_int4(u.game, u.nlvl, u.rng, u.flags | (nw << 8));
            q[2 * k + 1] = make_int4(qv[k], u.parent, u.nchild, w0);
        }
        int4 *pq;
        TRY(upload(c, &pq, q));
        *out = pq;
        return CFR_OK;
    };
    TRY(queue(H.up_queue, H.units, true, &d.upq));
    TRY(queue(H.down_queue, H.dunits, false, &d.downq));
    TRY(upload(c, &p32, H.game_root));
    d.game_root = p32;
    TRY(upload(c, &B.ext_inf, H.ext_inf));
    TRY(upload(c, &B.ext_seq0, H.ext_seq0));
    d.n_units = (int32_t)H.dunits.size();
    d.n_up = (int32_t)H.up_queue.size();
    d.G = (int32_t)L.G;
    TRY(dalloc(c, &d.r, H.S));
    TRY(dalloc(c, &d.b, H.S));
    TRY(dalloc(c, &d.x, H.S));
    TRY(dalloc(c, &d.xanc, H.xanc_size));
    d.fp64 = c->fp64 ? 1 : 0;
    d.r64 = d.b64 = d.x64 = d.xbar64 = d.evc64 = d.xanc64 = nullptr;
    if (c->fp64) {
        TRY(dalloc(c, &d.r64, H.S));
        TRY(dalloc(c, &d.b64, H.S));
        TRY(dalloc(c, &d.x64, H.S));
        TRY(dalloc(c, &d.xbar64, H.S));
        TRY(dalloc(c, &d.evc64, H.J));
        TRY(dalloc(c, &d.xanc64, H.xanc_size));
        for (double *a : {d.r64, d.x64, d.xbar64}) CU(cudaMemsetAsync(a, 0, H.S * sizeof(double), c->stream));
        CU(cudaMemsetAsync(d.evc64, 0, H.J * sizeof(double), c->stream));
    }
    TRY(dalloc(c, &d.xbar, H.S));
    TRY(dalloc(c, &d.u, H.S));
    TRY(dalloc(c, &d.ev, H.J));
    TRY(dalloc(c, &d.u64, H.S));
    TRY(dalloc(c, &d.ev64, H.J));
    TRY(dalloc(c, &d.xnorm, H.S));
    int32_t *ctr;
    const int64_t nu = (int64_t)H.units.size();
    TRY(dalloc(c, &ctr, nu + 12));
    CU(cudaMemsetAsync(ctr, 0, (nu + 12) * sizeof(int32_t), c->stream));
    d.unit_cnt = ctr;
    d.qup = ctr + nu;
    d.qdn = ctr + nu + 4;
    d.qavg = ctr + nu + 8;
    d.S = (int32_t)H.S;
    d.err = c->err;
    d.wait_ns = c->wait_ns;
    TRY(dalloc(c, &d.root_done, L.G));
    CU(cudaMemsetAsync(d.root_done, 0, L.G * sizeof(int32_t), c->stream));
    CU(cudaMemsetAsync(d.r, 0, H.S * sizeof(float2), c->stream));
    CU(cudaMemsetAsync(d.xbar, 0, H.S * sizeof(float2), c->stream));
    CU(cudaMemsetAsync(d.ev, 0, H.J * sizeof(float), c->stream));
    CU(cudaMemsetAsync(d.ev64, 0, H.J * sizeof(double), c->stream));
    CU(cudaMemsetAsync(d.x, 0, H.S * sizeof(float), c->stream));
    B.smem_br = (size_t)(kThreads / 32) * 32 * kStage * sizeof(double);
    const StagedConfig &cf = kConfigs[c->cfg];
    // the pass kernels overlap one another's tails: one shared-memory carve-out
    // for all of them, so that an SM that ran one kernel's CTAs takes the next
    // kernel's full count without first draining
    for (const void *fn : {(const void *)cf.up, (const void *)cf.down, (const void *)cf.half}) {
        CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_staged));
        CU(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
    }
    TRY(occupancy_grid((const void *)cf.up, c->threads, c->smem_staged, B.n_up, &B.grid_up));
    TRY(occupancy_grid((const void *)k_up<MODE_BR>, kThreads, B.smem_br, B.n_up, &B.grid_up_br));
    // the FP64 iteration's bottom-up CTAs also run the average update: as
    // many as fit, whatever the unit count
    TRY(occupancy_grid((const void *)k_up<MODE_CFR64>, kThreads, B.smem_br, INT32_MAX, &B.grid_up64));
    TRY(occupancy_grid((const void *)k_down64, kThreads, 0, B.n_units, &B.grid_down64));
    TRY(occupancy_grid((const void *)cf.down, c->threads, c->smem_staged, B.n_units, &B.grid_down));
    TRY(occupancy_grid((const void *)cf.half, c->threads, c->smem_staged, std::max(B.n_up, B.n_units),
                       &B.grid_half));
    k_uniform<<<(unsigned)std::min<int64_t>((H.J + kThreads - 1) / kThreads, 65535), kThreads, 0, c->stream>>>(d,
                                                                                                             H.J);
    CU(cudaGetLastError());
    return CFR_OK;
}

int load(const cfr_tree_desc *games, int64_t n, void *stream, const cfr_load_options *lo, cfr_ctx **out) {
    if (!out) return set_err(CFR_ERR_ARG, "out is NULL");
    *out = nullptr;
    int shape = -1;   // the library's choice, once the games are known
    bool flat = false;
    int passes = 0;
    bool values = false;
    uint64_t wait_ns = kFlagWaitNs;
    bool fp64 = false;
    if (lo) {
        if (lo->shape < 0 || lo->shape > kNumConfigs) return set_err(CFR_ERR_ARG, "unknown launch shape");
        if (lo->flat != 0 && lo->flat != 1) return set_err(CFR_ERR_ARG, "flat must be 0 or 1");
        if (lo->passes < 0 || lo->passes > 2) return set_err(CFR_ERR_ARG, "passes must be 0, 1 or 2");
        if (lo->values != 0 && lo->values != 1) return set_err(CFR_ERR_ARG, "values must be 0 or 1");
        if (lo->wait_us < 0) return set_err(CFR_ERR_ARG, "wait_us must not be negative");
        if (lo->precision != 0 && lo->precision != 32 && lo->precision != 64)
            return set_err(CFR_ERR_ARG, "precision must be 0, 32 or 64");
        for (int k = 0; k < 2; k++)
            if (lo->reserved[k] != 0) return set_err(CFR_ERR_ARG, "reserved load options must be zero");
        if (lo->shape > 0) shape = lo->shape - 1;
        flat = lo->flat != 0;
        passes = lo->passes;
        values = lo->values != 0;
        if (lo->wait_us > 0) wait_ns = 1000ull * (uint64_t)lo->wait_us;
        fp64 = lo->precision == 64;
    }
    if (!games || n < 1) return set_err(CFR_ERR_ARG, "no games");
    std::vector<TreeView> tv(n);
    for (int64_t g = 0; g < n; g++) {
        const cfr_tree_desc &t = games[g];
        if (t.n_nodes < 1 || !t.parent || !t.kind || !t.infoset || !t.action || !t.chance_prob || !t.payoff_p1)
            return set_err(CFR_ERR_ARG, "game " + std::to_string(g) + ": NULL array or empty tree");
        tv[g] = {t.n_nodes, t.parent, t.kind, t.infoset, t.action, t.chance_prob, t.payoff_p1};
    }
    if (shape < 0) {
        int64_t nodes = 0;
        for (int64_t g = 0; g < n; g++) nodes += games[g].n_nodes;
        shape = pick_config(n, nodes);
    }
    Layout L;
    std::string err;
    int rc;
    CompileOptions opt;
    {
        int dev = 0, sms = 148;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        const StagedConfig &cf = kConfigs[shape];
        opt.slots = std::max(1, sms) * cf.ctas_per_sm;
        opt.item_bytes = cf.item_bytes;
        opt.flat = flat;
    }
    try {
        rc = compile_forest(tv.data(), n, opt, &L, &err);
    } catch (const std::bad_alloc &) {
        return set_err(CFR_ERR_OOM, "host allocation failed while compiling");
    } catch (const std::exception &e) {
        return set_err(CFR_ERR_INVALID, e.what());
    }
    if (rc != ST_OK) return set_err(rc == ST_OOM ? CFR_ERR_OOM : CFR_ERR_INVALID, err);
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    cfr_ctx *c = new (std::nothrow) cfr_ctx();
    if (!c) return set_err(CFR_ERR_OOM, "context allocation");
    auto bail = [&](int code) {
        cfr_free(c);
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(set_err(CFR_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e)));
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(set_err(CFR_ERR_CUDA, cudaGetErrorString(e)));
        c->own_stream = true;
    }
    c->G = L.G;
    c->Z = L.Z;
    c->cfg = shape;
    c->split = passes != 1;
    c->values = values;
    c->wait_ns = wait_ns;
    c->fp64 = fp64;
    c->threads = kConfigs[c->cfg].threads;
    c->item_bytes = (int)opt.item_bytes;
    // two unit buffers; a unit too large to stage uses its buffer as the
    // payoff-product stage of the global-memory path
    c->smem_staged = 2 * (size_t)c->item_bytes;
    if ((rc = dalloc(c, &c->err, 1))) return bail(rc);
    if (cudaMemsetAsync(c->err, 0, sizeof(int32_t), c->stream) != cudaSuccess)
        return bail(set_err(CFR_ERR_CUDA, "memset"));
    c->game_nodes = L.game_nodes;
    c->game_nnz = L.game_nnz;
    for (int p = 0; p < 2; p++)
        if ((rc = build_player(c, L, p))) return bail(rc);
    if ((rc = dalloc(c, &c->t_done, L.G))) return bail(rc);
    if ((rc = dalloc(c, &c->active, L.G))) return bail(rc);
    if ((rc = dalloc(c, &c->active_keep, L.G))) return bail(rc);
    if ((rc = dalloc(c, &c->par, L.G * (kParamSpan + 1)))) return bail(rc);
    if (c->fp64 && (rc = dalloc(c, &c->par64, L.G * (kParamSpan + 1)))) return bail(rc);
    if ((rc = dalloc(c, &c->pbase, L.G))) return bail(rc);
    if ((rc = dalloc(c, &c->mixed, 1))) return bail(rc);
    if ((rc = dalloc(c, &c->br[0], L.G))) return bail(rc);
    if ((rc = dalloc(c, &c->br[1], L.G))) return bail(rc);
    int64_t smax = 0;
    for (int p = 0; p < 2; p++)
        for (int64_t g = 0; g < L.G; g++) smax = std::max<int64_t>(smax, L.pl[p].game_S[g]);
    c->scratch_n = smax + 1;
    if ((rc = dalloc(c, &c->scratch, 3 * c->scratch_n))) return bail(rc);
    c->active_host.assign(L.G, 1);
    if (cudaMemsetAsync(c->t_done, 0, L.G * sizeof(int32_t), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->active, 1, L.G, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->active_keep, 1, L.G, c->stream) != cudaSuccess)
        return bail(set_err(CFR_ERR_CUDA, "memset"));
    for (int p = 0; p < 2; p++)
        if ((rc = launch_rebuild_x(c, p))) return bail(rc);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(set_err(CFR_ERR_CUDA, cudaGetErrorString(e)));
    *out = c;
    return CFR_OK;
}

bool default_alternating(int variant) { return variant != CFR_VANILLA; }

// read the device error word after the stream has drained; a bounded device
// wait that gave up leaves the context unusable
int check_err(cfr_ctx *c) {
    if (c->poisoned) return set_err(CFR_ERR_STATE, "context unusable after an earlier device timeout");
    int32_t e = 0;
    CU(cudaMemcpyAsync(&e, c->err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (e) {
        c->poisoned = true;
        return set_err(CFR_ERR_TIMEOUT, "a bounded device wait gave up (a copy or a parent unit did not complete)");
    }
    return CFR_OK;
}

// The CUDA graph of K = key.k iterations for key's variant and parameters:
// captured and instantiated on first use, then kept by the context.
int graph_for(cfr_ctx *c, const GraphKey &key, bool alt, cudaGraphExec_t *out) {
    auto f = c->graphs.find(key);
    if (f != c->graphs.end()) {
        *out = f->second;
        return CFR_OK;
    }
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = CFR_OK;
    int64_t nk = 0;
    for (int k = 0; k < key.k && rc == CFR_OK; k++)
        rc = launch_iteration(c, key.variant, key.a, key.b, key.g, alt, k, &nk);
    cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ee != cudaSuccess) return set_err(CFR_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
    ee = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ee != cudaSuccess) return set_err(CFR_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ee));
    // the graph's device-side set-up now, not on its first replay
    ee = cudaGraphUpload(exec, c->stream);
    if (ee != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return set_err(CFR_ERR_CUDA, std::string("graph upload: ") + cudaGetErrorString(ee));
    }
    c->graphs[key] = exec;
    c->graph_kernels[key] = nk;
    *out = exec;
    return CFR_OK;
}

bool default_alternating(int variant);

int iterate(cfr_ctx *c, int64_t n, int variant, double alpha, double beta, double gamma) {
    if (!c) return set_err(CFR_ERR_ARG, "ctx is NULL");
    if (c->poisoned) return set_err(CFR_ERR_STATE, "context unusable after an earlier device timeout");
    if (n < 0) return set_err(CFR_ERR_ARG, "negative iteration count");
    if (variant < 0 || variant > 4) return set_err(CFR_ERR_ARG, "unknown variant");
    if (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(gamma))
        return set_err(CFR_ERR_ARG, "alpha, beta, gamma must be finite");
    const bool alt = c->update_mode == CFR_UPDATES_DEFAULT ? default_alternating(variant)
                                                           : c->update_mode == CFR_UPDATES_ALTERNATING;
    const int K = c->graph_k;
    int64_t done = 0;
    if (n >= K) {
        GraphKey key{variant, alt ? 2 : 1, K, alpha, beta, gamma};
        cudaGraphExec_t exec = nullptr;
        TRY(graph_for(c, key, alt, &exec));
        const int64_t nk = c->graph_kernels[key];
        for (; done + K <= n; done += K) {
            CU(cudaGraphLaunch(exec, c->stream));
            c->launches += nk;
        }
    }
    for (int64_t k = 0; done < n; done++, k++)
        TRY(launch_iteration(c, variant, alpha, beta, gamma, alt, (int)k, &c->launches));
    return CFR_OK;
}

int check_game(cfr_ctx *c, int64_t g, int player) {
    if (!c) return set_err(CFR_ERR_ARG, "ctx is NULL");
    if (g < 0 || g >= c->G) return set_err(CFR_ERR_ARG, "game index out of range");
    if (player != 1 && player != 2) return set_err(CFR_ERR_ARG, "player must be 1 or 2");
    return CFR_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// exploitability without allocating: scratch in a fixed device array
// ---------------------------------------------------------------------------
namespace {

// Best-response values of both players for up to kNoAllocMaxGames games.  Every
// GPU that loads this library holds the array (1 MiB) until the process exits.
constexpr int64_t kNoAllocMaxGames = 1 << 16;
static __device__ __align__(256) double g_noalloc_br[2 * kNoAllocMaxGames];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in.
int noalloc_scratch(int dev, double **out) {
    if (dev < 0 || dev >= kMaxDevices) return set_err_static(CFR_ERR_ARG, "device ordinal out of range for the scratch table");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_br) != cudaSuccess)
            return set_err_static(CFR_ERR_CUDA, "cudaGetSymbolAddress of the exploitability scratch failed");
        g_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_noalloc_ptr[dev];
    return CFR_OK;
}

__global__ void k_expl_combine(const double *br1, const double *br2, int64_t G, double *expl) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x)
        expl[g] = 0.5 * (br1[g] + br2[g]);
}

}  // namespace

extern "C" {

int cfr_exploitability_batch_noalloc(cfr_ctx *ctx, double *dev_expl) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (!ctx) return set_err_static(CFR_ERR_ARG, "ctx is NULL");
    if (!dev_expl) return set_err_static(CFR_ERR_ARG, "dev_expl is NULL");
    if (ctx->poisoned) return set_err_static(CFR_ERR_STATE, "context unusable after an earlier device timeout");
    if (ctx->G > kNoAllocMaxGames)
        return set_err_static(CFR_ERR_ARG, "too many games: the no-allocation exploitability handles at most 65536");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_err_static(CFR_ERR_CUDA, "cudaGetDevice failed");
    if (dev != ctx->device) return set_err_static(CFR_ERR_ARG, "the context's device must be current");
    double *br = nullptr;
    TRY(noalloc_scratch(dev, &br));
    double *br1 = br, *br2 = br + kNoAllocMaxGames;
    // the scratch keeps the previous call's values: start every game from NaN
    // (all bits set), so a game whose pass did not finish reads as NaN, never
    // as a stale or zero exploitability
    if (cudaMemsetAsync(br1, 0xFF, ctx->G * sizeof(double), ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(br2, 0xFF, ctx->G * sizeof(double), ctx->stream) != cudaSuccess)
        return set_err_static(CFR_ERR_CUDA, "clearing the exploitability scratch failed");
    const bool masked = std::find(ctx->active_host.begin(), ctx->active_host.end(), 0) != ctx->active_host.end();
    if (masked && cudaMemsetAsync(ctx->active, 1, ctx->G, ctx->stream) != cudaSuccess)
        return set_err_static(CFR_ERR_CUDA, "cudaMemsetAsync failed");
    DevGames gm{ctx->t_done, ctx->active, nullptr};
    IterArgs ia{};
    for (int p = 0; p < 2; p++) {
        PlayerBuf &B = ctx->pl[p];
        k_normalize<<<(unsigned)std::min<int64_t>((B.S + kThreads - 1) / kThreads, 65535), kThreads, 0,
                      ctx->stream>>>(B.d, B.S);
    }
    for (int p = 0; p < 2; p++) {
        PlayerBuf &B = ctx->pl[p];
        gm.br = p == 0 ? br1 : br2;
        ia.sign = p == 0 ? 1.f : -1.f;
        k_up<MODE_BR><<<B.grid_up_br, kThreads, B.smem_br, ctx->stream>>>(B.d, gm, ctx->pl[1 - p].d.xnorm, ia);
    }
    k_expl_combine<<<(unsigned)std::min<int64_t>((ctx->G + 255) / 256, 65535), 256, 0, ctx->stream>>>(br1, br2,
                                                                                                    ctx->G, dev_expl);
    if (cudaGetLastError() != cudaSuccess) return set_err_static(CFR_ERR_CUDA, "kernel launch failed");
    // the caller's mask back, from its device copy (no host memory involved)
    if (masked && cudaMemcpyAsync(ctx->active, ctx->active_keep, ctx->G, cudaMemcpyDeviceToDevice,
                                  ctx->stream) != cudaSuccess)
        return set_err_static(CFR_ERR_CUDA, "cudaMemcpyAsync failed");
    return CFR_OK;
}

int cfr_exploitability_async(cfr_ctx *ctx, double *dev_expl) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (!ctx) return set_err(CFR_ERR_ARG, "ctx is NULL");
    if (!dev_expl) return set_err(CFR_ERR_ARG, "dev_expl is NULL");
    if (ctx->poisoned) return set_err(CFR_ERR_STATE, "context unusable after an earlier device timeout");
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != ctx->device) return set_err(CFR_ERR_ARG, "the context's device must be current");
    double *br1 = ctx->br[0], *br2 = ctx->br[1];
    // a game whose best-response pass did not finish reads as NaN
    CU(cudaMemsetAsync(br1, 0xFF, ctx->G * sizeof(double), ctx->stream));
    CU(cudaMemsetAsync(br2, 0xFF, ctx->G * sizeof(double), ctx->stream));
    const bool masked = std::find(ctx->active_host.begin(), ctx->active_host.end(), 0) != ctx->active_host.end();
    if (masked) CU(cudaMemsetAsync(ctx->active, 1, ctx->G, ctx->stream));
    DevGames gm{ctx->t_done, ctx->active, nullptr};
    IterArgs ia{};
    for (int p = 0; p < 2; p++) {
        PlayerBuf &B = ctx->pl[p];
        k_normalize<<<(unsigned)std::min<int64_t>((B.S + kThreads - 1) / kThreads, 65535), kThreads, 0,
                      ctx->stream>>>(B.d, B.S);
    }
    for (int p = 0; p < 2; p++) {
        PlayerBuf &B = ctx->pl[p];
        gm.br = p == 0 ? br1 : br2;
        ia.sign = p == 0 ? 1.f : -1.f;
        k_up<MODE_BR><<<B.grid_up_br, kThreads, B.smem_br, ctx->stream>>>(B.d, gm, ctx->pl[1 - p].d.xnorm, ia);
    }
    k_expl_combine<<<(unsigned)std::min<int64_t>((ctx->G + 255) / 256, 65535), 256, 0, ctx->stream>>>(br1, br2,
                                                                                                    ctx->G, dev_expl);
    CU(cudaGetLastError());
    if (masked) CU(cudaMemcpyAsync(ctx->active, ctx->active_keep, ctx->G, cudaMemcpyDeviceToDevice, ctx->stream));
    return CFR_OK;
}

int cfr_copy_game_states(cfr_ctx *dst, int64_t n, const int64_t *host_dst_games, cfr_ctx *src,
                         const int64_t *host_src_games) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (!dst || !src || (n > 0 && (!host_dst_games || !host_src_games)))
        return set_err(CFR_ERR_ARG, "NULL context or game list");
    if (n < 0) return set_err(CFR_ERR_ARG, "negative game count");
    if (dst->poisoned || src->poisoned) return set_err(CFR_ERR_STATE, "context unusable after an earlier device timeout");
    if (dst == src) return set_err(CFR_ERR_ARG, "source and destination must differ");
    if (dst->device != src->device) return set_err(CFR_ERR_ARG, "both contexts must be on one device");
    if (dst->fp64 != src->fp64) return set_err(CFR_ERR_ARG, "both contexts must have the same precision");
    for (int64_t k = 0; k < n; k++) {
        const int64_t gd = host_dst_games[k], gs = host_src_games[k];
        if (gd < 0 || gd >= dst->G || gs < 0 || gs >= src->G) return set_err(CFR_ERR_ARG, "game index out of range");
        for (int p = 0; p < 2; p++)
            if (dst->pl[p].game_S[gd] != src->pl[p].game_S[gs] || dst->pl[p].game_J[gd] != src->pl[p].game_J[gs])
                return set_err(CFR_ERR_ARG, "games differ in their sequence or infoset counts");
        if (dst->game_nodes[gd] != src->game_nodes[gs] || dst->game_nnz[gd] != src->game_nnz[gs])
            return set_err(CFR_ERR_ARG, "games differ in their node or payoff counts");
    }
    if (n == 0) return CFR_OK;
    // the source's work so far comes first
    cudaEvent_t ev = nullptr;
    CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, src->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(dst->stream, ev, 0);
    cudaEventDestroy(ev);
    CU(e);
    for (int64_t k = 0; k < n; k++) {
        const int64_t gd = host_dst_games[k], gs = host_src_games[k];
        for (int p = 0; p < 2; p++) {
            PlayerBuf &D = dst->pl[p], &S = src->pl[p];
            const int Jg = D.game_J[gd];
            k_copy_game<<<(Jg + kThreads) / kThreads, kThreads, 0, dst->stream>>>(
                D.d, D.ext_inf + D.game_jbase[gd], (int)gd, S.d, S.ext_inf + S.game_jbase[gs], (int)gs, Jg);
        }
        k_copy_t<<<1, 1, 0, dst->stream>>>(dst->t_done, (int)gd, src->t_done, (int)gs);
    }
    CU(cudaGetLastError());
    for (int p = 0; p < 2; p++) TRY(launch_rebuild_x(dst, p));
    // the source may be freed once this returns
    CU(cudaStreamSynchronize(dst->stream));
    return check_err(dst);
}

int cfr_load_tree(const cfr_tree_desc *tree, void *cuda_stream, cfr_ctx **out) {
    return load(tree, 1, cuda_stream, nullptr, out);
}

int cfr_load_batch(const cfr_tree_desc *games, int64_t n_games, void *cuda_stream, cfr_ctx **out) {
    return load(games, n_games, cuda_stream, nullptr, out);
}

int cfr_load_batch_opts(const cfr_tree_desc *games, int64_t n_games, void *cuda_stream,
                        const cfr_load_options *options, cfr_ctx **out) {
    return load(games, n_games, cuda_stream, options, out);
}

int cfr_num_shapes(void) { return kNumConfigs; }

int cfr_default_shape(void) { return kDefaultConfig + 1; }

int cfr_pick_shape(int64_t n_games, int64_t total_nodes) {
    if (n_games < 1 || total_nodes < 1) return set_err_static(CFR_ERR_ARG, "n_games and total_nodes must be positive");
    return pick_config(n_games, total_nodes) + 1;
}

int cfr_shape_info(int shape, int32_t *host_out3) {
    if (!host_out3) return set_err(CFR_ERR_ARG, "host_out3 is NULL");
    if (shape < 1 || shape > kNumConfigs) return set_err(CFR_ERR_ARG, "unknown launch shape");
    const StagedConfig &cf = kConfigs[shape - 1];
    host_out3[0] = cf.threads;
    host_out3[1] = cf.ctas_per_sm;
    host_out3[2] = cf.item_bytes;
    return CFR_OK;
}

int cfr_iterate(cfr_ctx *ctx, int64_t n, cfr_variant v, double alpha, double beta, double gamma) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (ctx && std::find(ctx->active_host.begin(), ctx->active_host.end(), 0) != ctx->active_host.end()) {
        std::fill(ctx->active_host.begin(), ctx->active_host.end(), 1);
        CU(cudaMemsetAsync(ctx->active, 1, ctx->G, ctx->stream));
        CU(cudaMemsetAsync(ctx->active_keep, 1, ctx->G, ctx->stream));
    }
    return iterate(ctx, n, (int)v, alpha, beta, gamma);
}

int cfr_iterate_batch(cfr_ctx *ctx, int64_t n, cfr_variant v, double alpha, double beta, double gamma,
                      const uint8_t *host_active) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (!ctx) return set_err(CFR_ERR_ARG, "ctx is NULL");
    std::vector<uint8_t> act(ctx->G, 1);
    if (host_active)
        for (int64_t g = 0; g < ctx->G; g++) act[g] = host_active[g] ? 1 : 0;
    if (act != ctx->active_host) {
        ctx->active_host = act;
        // pageable source: the copy is staged before the call returns
        CU(cudaMemcpyAsync(ctx->active, ctx->active_host.data(), ctx->G, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(ctx->active_keep, ctx->active, ctx->G, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return iterate(ctx, n, (int)v, alpha, beta, gamma);
}

int cfr_prepare_graph(cfr_ctx *ctx, cfr_variant v, double alpha, double beta, double gamma) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (!ctx) return set_err(CFR_ERR_ARG, "ctx is NULL");
    if (ctx->poisoned) return set_err(CFR_ERR_STATE, "context unusable after an earlier device timeout");
    if ((int)v < 0 || (int)v > 4) return set_err(CFR_ERR_ARG, "unknown variant");
    if (!std::isfinite(alpha) || !std::isfinite(beta) || !std::isfinite(gamma))
        return set_err(CFR_ERR_ARG, "alpha, beta, gamma must be finite");
    const bool alt = ctx->update_mode == CFR_UPDATES_DEFAULT ? default_alternating((int)v)
                                                             : ctx->update_mode == CFR_UPDATES_ALTERNATING;
    GraphKey key{(int)v, alt ? 2 : 1, ctx->graph_k, alpha, beta, gamma};
    cudaGraphExec_t exec = nullptr;
    return graph_for(ctx, key, alt, &exec);
}

int cfr_set_update_mode(cfr_ctx *ctx, int mode) {
    if (!ctx) return set_err(CFR_ERR_ARG, "ctx is NULL");
    if (mode < 0 || mode > 2) return set_err(CFR_ERR_ARG, "unknown update mode");
    ctx->update_mode = mode;
    return CFR_OK;
}

int cfr_set_graph_iterations(cfr_ctx *ctx, int k) {
    if (!ctx) return set_err(CFR_ERR_ARG, "ctx is NULL");
    if (k < 1 || k > 4096) return set_err(CFR_ERR_ARG, "graph iterations must be in [1, 4096]");
    ctx->graph_k = k;
    return CFR_OK;
}

int cfr_sizes(cfr_ctx *ctx, int64_t game, int64_t *out) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    TRY(check_game(ctx, game, 1));
    if (!out) return set_err(CFR_ERR_ARG, "out is NULL");
    int32_t t = 0;
    CU(cudaMemcpyAsync(&t, ctx->t_done + game, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    out[0] = ctx->pl[0].game_S[game];
    out[1] = ctx->pl[1].game_S[game];
    out[2] = ctx->pl[0].game_J[game];
    out[3] = ctx->pl[1].game_J[game];
    out[4] = ctx->game_nnz[game];
    out[5] = ctx->game_nodes[game];
    out[6] = t;
    out[7] = ctx->G;
    out[8] = ctx->dev_bytes;
    out[9] = ctx->h2d_bytes;
    return CFR_OK;
}

int cfr_get_average_strategy(cfr_ctx *ctx, int64_t game, int player, double *host_out, int64_t len) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    TRY(check_game(ctx, game, player));
    PlayerBuf &B = ctx->pl[player - 1];
    const int Jg = B.game_J[game];
    if (!host_out || len != B.game_S[game]) return set_err(CFR_ERR_ARG, "output length must equal S_p");
    if (Jg > 0) {
        k_average<<<(Jg + kThreads - 1) / kThreads, kThreads, 0, ctx->stream>>>(
            B.d, B.ext_inf + B.game_jbase[game], B.ext_seq0 + B.game_jbase[game], Jg, ctx->scratch);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(host_out, ctx->scratch, len * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    return check_err(ctx);
}

int cfr_exploitability_batch(cfr_ctx *ctx, double *host_expl, double *host_br1, double *host_br2) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (!ctx) return set_err(CFR_ERR_ARG, "ctx is NULL");
    if (ctx->poisoned) return set_err(CFR_ERR_STATE, "context unusable after an earlier device timeout");
    DevGames gm{ctx->t_done, ctx->active, nullptr};
    IterArgs ia{};
    // the best response is computed for every game, whatever the active mask
    const bool masked = std::find(ctx->active_host.begin(), ctx->active_host.end(), 0) != ctx->active_host.end();
    if (masked) CU(cudaMemsetAsync(ctx->active, 1, ctx->G, ctx->stream));
    for (int p = 0; p < 2; p++) {
        PlayerBuf &B = ctx->pl[p];
        k_normalize<<<(unsigned)std::min<int64_t>((B.S + kThreads - 1) / kThreads, 65535), kThreads, 0,
                      ctx->stream>>>(B.d, B.S);
    }
    for (int p = 0; p < 2; p++) {
        PlayerBuf &B = ctx->pl[p];
        gm.br = ctx->br[p];
        ia.sign = p == 0 ? 1.f : -1.f;
        k_up<MODE_BR><<<B.grid_up_br, kThreads, B.smem_br, ctx->stream>>>(B.d, gm, ctx->pl[1 - p].d.xnorm, ia);
    }
    CU(cudaGetLastError());
    if (masked) CU(cudaMemcpyAsync(ctx->active, ctx->active_keep, ctx->G, cudaMemcpyDeviceToDevice, ctx->stream));
    std::vector<double> b1(ctx->G), b2(ctx->G);
    CU(cudaMemcpyAsync(b1.data(), ctx->br[0], ctx->G * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(b2.data(), ctx->br[1], ctx->G * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    TRY(check_err(ctx));
    for (int64_t g = 0; g < ctx->G; g++) {
        if (host_expl) host_expl[g] = 0.5 * (b1[g] + b2[g]);
        if (host_br1) host_br1[g] = b1[g];
        if (host_br2) host_br2[g] = b2[g];
    }
    return CFR_OK;
}

int cfr_exploitability(cfr_ctx *ctx, double *expl, double *br1, double *br2) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (!ctx) return set_err(CFR_ERR_ARG, "ctx is NULL");
    std::vector<double> e(ctx->G), a(ctx->G), b(ctx->G);
    TRY(cfr_exploitability_batch(ctx, e.data(), a.data(), b.data()));
    if (expl) *expl = e[0];
    if (br1) *br1 = a[0];
    if (br2) *br2 = b[0];
    return CFR_OK;
}

int cfr_get_state(cfr_ctx *ctx, int64_t game, int player, double *host_r, double *host_b, double *host_xbar,
                  int64_t *t) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    TRY(check_game(ctx, game, player));
    PlayerBuf &B = ctx->pl[player - 1];
    const int Jg = B.game_J[game];
    const int64_t Sg = B.game_S[game];
    double *dr = ctx->scratch, *db = ctx->scratch + ctx->scratch_n, *dx = ctx->scratch + 2 * ctx->scratch_n;
    k_get_state<<<(Jg + kThreads) / kThreads, kThreads, 0, ctx->stream>>>(
        B.d, B.ext_inf + B.game_jbase[game], B.ext_seq0 + B.game_jbase[game], (int)game, Jg, dr, db, dx);
    CU(cudaGetLastError());
    if (host_r && Sg) CU(cudaMemcpyAsync(host_r, dr, Sg * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (host_b && Sg) CU(cudaMemcpyAsync(host_b, db, Sg * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (host_xbar) CU(cudaMemcpyAsync(host_xbar, dx, (Sg + 1) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    int32_t tt = 0;
    CU(cudaMemcpyAsync(&tt, ctx->t_done + game, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    TRY(check_err(ctx));
    if (t) *t = tt;
    return CFR_OK;
}

int cfr_get_values(cfr_ctx *ctx, int64_t game, int player, double *host_x, double *host_ev) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    TRY(check_game(ctx, game, player));
    if (!ctx->values) return set_err(CFR_ERR_STATE, "load the context with the values option to read values");
    PlayerBuf &B = ctx->pl[player - 1];
    const int Jg = B.game_J[game];
    const int64_t Sg = B.game_S[game];
    // the transfer area holds 3 (max S + 1) doubles: x in the first part, ev
    // (J <= S) in the second
    double *dx = ctx->scratch, *de = ctx->scratch + ctx->scratch_n;
    k_get_values<<<(Jg + kThreads) / kThreads, kThreads, 0, ctx->stream>>>(
        B.d, B.ext_inf + B.game_jbase[game], B.ext_seq0 + B.game_jbase[game], (int)game, Jg, dx, de);
    CU(cudaGetLastError());
    if (host_x) CU(cudaMemcpyAsync(host_x, dx, (Sg + 1) * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (host_ev && Jg) CU(cudaMemcpyAsync(host_ev, de, Jg * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return check_err(ctx);
}

int cfr_set_state(cfr_ctx *ctx, int64_t game, int player, const double *host_r, const double *host_b,
                  const double *host_xbar, int64_t t) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    TRY(check_game(ctx, game, player));
    if (!host_r || !host_b || !host_xbar) return set_err(CFR_ERR_ARG, "state arrays must not be NULL");
    if (t < 0 || t > INT32_MAX - 1) return set_err(CFR_ERR_ARG, "t out of range");
    PlayerBuf &B = ctx->pl[player - 1];
    const int Jg = B.game_J[game];
    const int64_t Sg = B.game_S[game];
    double *dr = ctx->scratch, *db = ctx->scratch + ctx->scratch_n, *dx = ctx->scratch + 2 * ctx->scratch_n;
    if (Sg) {
        CU(cudaMemcpyAsync(dr, host_r, Sg * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(db, host_b, Sg * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    }
    CU(cudaMemcpyAsync(dx, host_xbar, (Sg + 1) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    k_set_state<<<(Jg + kThreads) / kThreads, kThreads, 0, ctx->stream>>>(
        B.d, B.ext_inf + B.game_jbase[game], B.ext_seq0 + B.game_jbase[game], (int)game, Jg, dr, db, dx);
    k_set_t<<<1, 1, 0, ctx->stream>>>(ctx->t_done, (int)game, (int32_t)t);
    CU(cudaGetLastError());
    TRY(launch_rebuild_x(ctx, player - 1));
    CU(cudaStreamSynchronize(ctx->stream));
    return check_err(ctx);
}

int cfr_profile_iterations(cfr_ctx *ctx, int64_t n, cfr_variant v, double alpha, double beta, double gamma,
                           float *host_ms) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (!ctx) return set_err(CFR_ERR_ARG, "ctx is NULL");
    if (!host_ms || n < 1) return set_err(CFR_ERR_ARG, "need n >= 1 and an output array");
    if ((int)v < 0 || (int)v > 4) return set_err(CFR_ERR_ARG, "unknown variant");
    const bool alt = ctx->update_mode == CFR_UPDATES_DEFAULT ? default_alternating((int)v)
                                                             : ctx->update_mode == CFR_UPDATES_ALTERNATING;
    cudaEvent_t ev[5];
    for (int k = 0; k < 5; k++) CU(cudaEventCreate(&ev[k]));
    double tot[4] = {0, 0, 0, 0};
    int rc = CFR_OK;
    for (int64_t i = 0; i < n && rc == CFR_OK; i++) {
        rc = launch_iteration(ctx, (int)v, alpha, beta, gamma, alt, (int)i, &ctx->launches, ev);
        if (rc) break;
        cudaError_t e = cudaEventSynchronize(ev[4]);
        if (e != cudaSuccess) {
            rc = set_err(CFR_ERR_CUDA, cudaGetErrorString(e));
            break;
        }
        for (int k = 0; k < 4; k++) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            tot[k] += ms;
        }
    }
    for (int k = 0; k < 5; k++) cudaEventDestroy(ev[k]);
    for (int k = 0; k < 4; k++) host_ms[k] = (float)tot[k];
    if (rc) return rc;
    return check_err(ctx);
}

int cfr_kernel_launches(cfr_ctx *ctx, int64_t *host_count) {
    if (!ctx || !host_count) return set_err(CFR_ERR_ARG, "ctx and host_count must not be NULL");
    *host_count = ctx->launches;
    return CFR_OK;
}

int cfr_sync(cfr_ctx *ctx) {
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (!ctx) return set_err(CFR_ERR_ARG, "ctx is NULL");
    CU(cudaStreamSynchronize(ctx->stream));
    return check_err(ctx);
}

void cfr_free(cfr_ctx *ctx) {
    if (!ctx) return;
    std::lock_guard<std::recursive_mutex> setup(setup_mutex());
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    for (void *p : ctx->allocs) cudaFree(p);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *cfr_strerror(int status) {
    switch (status) {
        case CFR_OK: return "ok";
        case CFR_ERR_INVALID: return "invalid game tree";
        case CFR_ERR_OOM: return "out of memory";
        case CFR_ERR_CUDA: return "CUDA error";
        case CFR_ERR_TIMEOUT: return "device wait timed out";
        case CFR_ERR_STATE: return "invalid state for this call";
        case CFR_ERR_ARG: return "invalid argument";
        default: return "unknown status";
    }
}

const char *cfr_last_error(void) { return g_last_error_static ? g_last_error_static : g_last_error.c_str(); }

}  // extern "C"
