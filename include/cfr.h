/*
 * cfr.h -- C ABI of the B300 sequence-form CFR library (libcfr.so).
 *
 * The library runs the hot path of "Parallelizing Counterfactual Regret
 * Minimization" (Kim & Sandholm): sequence-form CFR (Sec. 2.1, Alg. 1) written
 * as passes over a flattened game tree (Alg. 2), with the CFR+, DCFR and PCFR+
 * variants (Alg. 3-5) and alternating updates (Sec. 3.5.1), for two-player
 * zero-sum extensive-form games with perfect recall.  Every step runs in CUDA
 * kernels on the current device; there is no CPU fallback.  Best response and
 * exploitability run in FP64 on the GPU.
 *
 * Conventions for every call:
 *   - All functions return an int status: CFR_OK (0) or a negative CFR_ERR_*.
 *     No call aborts the process and no C++ exception crosses this boundary.
 *   - The library copies every input it is given; output buffers belong to the
 *     caller.  Buffers named host_* are host memory; the only device pointer in
 *     this ABI is the output of cfr_exploitability_batch_noalloc.
 *   - All device work of a context is issued on the CUDA stream passed at load
 *     time (a cudaStream_t given as void*; NULL = a non-blocking stream the
 *     context creates and owns).  Calls that return data synchronise that
 *     stream before returning.
 *   - Sequence-indexed vectors are in the caller's (infoset id, action) order:
 *     player p's sequence k is action a of caller infoset j where
 *     k = sum_{j' < j} |A_j'| + a.  Average-sum vectors (xbar) carry the empty
 *     sequence first: xbar[0] = empty, xbar[1 + k] = sequence k.
 *   - Not thread-safe per context: one host thread at a time per context.
 */
#ifndef CFR_B300_H
#define CFR_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CFR_OK 0
#define CFR_ERR_INVALID (-1)   /* malformed tree: see cfr_last_error() */
#define CFR_ERR_OOM (-2)       /* device or host allocation failed */
#define CFR_ERR_CUDA (-3)      /* a CUDA call failed (message in cfr_last_error()) */
#define CFR_ERR_TIMEOUT (-4)   /* a bounded device wait gave up; the context is unusable */
#define CFR_ERR_STATE (-5)     /* call not valid in the context's current state */
#define CFR_ERR_ARG (-6)       /* bad argument (NULL pointer, length, index, variant) */

/* regret-minimiser variants (Sec. 2.1, Alg. 1, Alg. 3, Alg. 4, Alg. 5) */
typedef enum {
    CFR_VANILLA = 0,    /* regret matching */
    CFR_PLUS = 1,       /* regret matching+ : r := r^+ after ObserveUtility (Alg. 3) */
    CFR_DCFR = 2,       /* discounted: r *= t^a/(t^a+1) where r>0, t^b/(t^b+1) where r<0 (Alg. 4) */
    CFR_PCFR_PLUS = 3,  /* predictive RM+ with prediction m^t = u^(t-1) (Alg. 5) */
    CFR_PCFR = 4        /* predictive RM, regrets never floored (Alg. 5, Sec. 3.5.4) */
} cfr_variant;

/* update schedule (Sec. 3.5.1) */
#define CFR_UPDATES_DEFAULT 0       /* vanilla: simultaneous; the other variants: alternating */
#define CFR_UPDATES_SIMULTANEOUS 1
#define CFR_UPDATES_ALTERNATING 2

/* A game tree, flat.  Node 0 is the root and every parent precedes its
 * children (parent[i] < i).  Node kinds: 0 chance, 1 player-1 decision,
 * 2 player-2 decision, 3 terminal.  Decision nodes carry an infoset id, dense
 * 0..J_p-1 per player; all nodes of an infoset must have the same number of
 * children and the same parent sequence (perfect recall).  action[i] is the
 * index (0..children-1) of the edge from parent[i] to i.  chance_prob[i] is the
 * probability of that edge when the parent is a chance node (ignored
 * otherwise); payoff_p1[i] is player 1's utility at terminal i (player 2 gets
 * the negative).  The arrays are host memory, read during the call only. */
typedef struct {
    int64_t n_nodes;
    const int32_t *parent;
    const int8_t *kind;
    const int32_t *infoset;
    const int32_t *action;
    const double *chance_prob;
    const double *payoff_p1;
} cfr_tree_desc;

typedef struct cfr_ctx cfr_ctx;   /* opaque; owns all its device memory */

/* Compile a tree (Sec. 2.1 sequence form, Sec. 3.1-3.2 logic matrices and
 * level graphs as index arrays) and upload it.  Validates the tree
 * (CFR_ERR_INVALID with a message on imperfect recall, action-count
 * mismatches, chance probabilities not summing to 1, non-finite payoffs,
 * bad ordering).  The initial state is r = 0, uniform strategies, t = 0.
 * On success *out owns the context; free it with cfr_free(). */
int cfr_load_tree(const cfr_tree_desc *tree, void *cuda_stream, cfr_ctx **out);

/* Same for n_games independent games sharing one context ("batch"): every
 * kernel launch advances all active games together.  Game g keeps its own
 * iteration counter.  games: host array of n_games descriptors. */
int cfr_load_batch(const cfr_tree_desc *games, int64_t n_games, void *cuda_stream, cfr_ctx **out);

/* Layout and launch choices made at load time.  All zero selects the
 * library's defaults.
 *   shape: 0 = default, k >= 1 = launch shape k of cfr_shape_info (threads per
 *          CTA, CTAs per SM, unit buffer bytes); the units of work are sized
 *          for the shape.
 *   flat:  1 = one tree level per unit below a root unit that holds the narrow
 *          top of each game; 0 = several levels per unit (default).
 *   passes: how the alternating schedule launches one player's bottom-up
 *          and top-down passes.  1 = one kernel, in which the top-down units
 *          of a game start as soon as that game's bottom-up pass is complete;
 *          2 = two kernels; 0 = the library's choice (two kernels, the faster
 *          on the workloads measured).
 *   values: 1 = every bottom-up pass also stores the expected counterfactual
 *          value ev_j of every infoset (Alg. 1 ObserveUtility), so that
 *          cfr_get_values can return them; 0 = only what the iteration needs
 *          (default; about 4 bytes per infoset less traffic per pass).
 *   wait_us: longest time, in microseconds, that a unit of work waits on the
 *          GPU for the units it depends on before giving up (the wait is
 *          bounded so that a fault elsewhere cannot hang the device; the
 *          context then reports CFR_ERR_TIMEOUT); 0 = the default, 1 s.
 *   precision: 0 or 32 = the passes in FP32 with float-float (Kahan)
 *          regret and average sums (default, the fast path); 64 = every
 *          pass in FP64 from global memory (payoffs, values, regrets,
 *          strategies and averages), for games whose iterates are sensitive
 *          to FP32 rounding or range (exact regret ties, reach below 1e-38);
 *          several times slower.  Calls that return state convert it to FP64
 *          either way.
 *   reserved: must be zero.
 * Every choice computes the same iteration; they differ only in speed (see
 * the autotuner in the Python package). */
typedef struct {
    int32_t shape;
    int32_t flat;
    int32_t passes;
    int32_t values;
    int32_t wait_us;
    int32_t precision;
    int32_t reserved[2];
} cfr_load_options;

/* cfr_load_batch with load options (NULL = defaults).  CFR_ERR_ARG on an
 * unknown shape, a flat or values field other than 0/1, passes outside 0..2,
 * a negative wait_us, a precision other than 0, 32 or 64, or a nonzero
 * reserved field. */
int cfr_load_batch_opts(const cfr_tree_desc *games, int64_t n_games, void *cuda_stream,
                        const cfr_load_options *options, cfr_ctx **out);

/* Number of launch shapes (shape indices 1..cfr_num_shapes()); the shape that
 * options.shape = 0 selects for a single game of at least 1M nodes
 * (cfr_default_shape); and the shape it selects for any load of n_games games
 * of total_nodes nodes in all (cfr_pick_shape: the default shape for one
 * game of at least 1M nodes, else the 256-thread, 3-CTA, 32 KB shape, which
 * runs batches and small games faster; CFR_ERR_ARG unless both counts are
 * positive). */
int cfr_num_shapes(void);
int cfr_default_shape(void);
int cfr_pick_shape(int64_t n_games, int64_t total_nodes);

/* Launch shape k: host_out3 = {threads per CTA, CTAs per SM, unit buffer
 * bytes}.  CFR_ERR_ARG for k outside 1..cfr_num_shapes(). */
int cfr_shape_info(int shape, int32_t *host_out3);

/* Run n iterations of the chosen variant on every game (Alg. 2 NextStrategy /
 * ObserveUtility per player; Alg. 3/4/5 post-ops).  alpha, beta: DCFR
 * exponents (ignored by the other variants).  gamma: average-strategy weight
 * exponent, xbar += t^gamma x^t for every variant (0 = uniform average).
 * Iterations continue from each game's stored counter: 10 calls of n = 100
 * equal one call of n = 1000.  Asynchronous on the context's stream. */
int cfr_iterate(cfr_ctx *ctx, int64_t n, cfr_variant v, double alpha, double beta, double gamma);

/* As cfr_iterate, advancing only the games whose host_active[g] is nonzero
 * (host_active: n_games bytes; NULL = all games). */
int cfr_iterate_batch(cfr_ctx *ctx, int64_t n, cfr_variant v, double alpha, double beta, double gamma,
                      const uint8_t *host_active);

/* Choose the update schedule (CFR_UPDATES_*). */
int cfr_set_update_mode(cfr_ctx *ctx, int mode);

/* Number of iterations captured per CUDA graph replay (1..4096, default 64). */
int cfr_set_graph_iterations(cfr_ctx *ctx, int k);

/* Capture and instantiate now the CUDA graph that cfr_iterate replays for
 * this variant and these parameters at the context's graph length (and
 * update schedule), without running it, so that the first cfr_iterate of at
 * least that many iterations only replays it.  Nothing is computed and no
 * state changes. */
int cfr_prepare_graph(cfr_ctx *ctx, cfr_variant v, double alpha, double beta, double gamma);

/* Sizes of game g: out[0..9] = S1, S2 (non-empty sequences), J1, J2
 * (infosets), nnz of the payoff matrix, game-tree nodes, completed
 * iterations, number of games in the context, device bytes the context holds,
 * bytes copied host-to-device when it was loaded. */
int cfr_sizes(cfr_ctx *ctx, int64_t game, int64_t *host_out10);

/* Average behavioural strategy of game g, player p (1 or 2), FP64:
 * xbar[(j,a)] / xbar[p_j], uniform where xbar[p_j] = 0.  len must be S_p. */
int cfr_get_average_strategy(cfr_ctx *ctx, int64_t game, int player, double *host_out, int64_t len);

/* Exploitability of the average profile of game 0, computed in FP64 on the
 * GPU: BR1 = max_x x^T M ybar, BR2 = max_y -xbar^T M y over the normalised
 * averages (current strategies when no iteration has run);
 * expl = (BR1 + BR2) / 2.  Any output pointer may be NULL. */
int cfr_exploitability(cfr_ctx *ctx, double *expl, double *br1, double *br2);

/* Same for every game of the context: host arrays of n_games entries each
 * (any may be NULL). */
int cfr_exploitability_batch(cfr_ctx *ctx, double *host_expl, double *host_br1, double *host_br2);

/* Exploitability of every game, like cfr_exploitability_batch, for callers
 * that cannot allocate memory at the point of the call: code running under a
 * memory manager that owns the whole device pool (a framework's caching
 * allocator, an embedded runtime with a fixed budget), or loops where the
 * device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.  The
 * paper has no counterpart; this is an interface variant of the FP64
 * best-response pass.
 *   - dev_expl: caller-owned DEVICE buffer of n_games doubles (the one device
 *     pointer of this ABI); expl[g] = (BR1 + BR2) / 2 as in
 *     cfr_exploitability_batch.
 *   - Allocates nothing (no cudaMalloc/cudaFree, no host heap): the per-game
 *     best-response values live in a fixed device array of the library that
 *     holds at most 65536 games (1 MiB, kept on every GPU that loads the
 *     library until the process exits).  Contexts with more games get
 *     CFR_ERR_ARG.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the context's device current; make that
 *     first call before any stream capture.
 *   - Asynchronous on the context's stream: dev_expl is valid once the stream
 *     has reached this point (e.g. after cfr_sync).  A game whose
 *     best-response pass gave up on a bounded wait reads as NaN; the timeout
 *     status itself is reported only by the next synchronising call
 *     (cfr_sync and the calls that return data).  All calls share the one
 *     array, so calls whose work overlaps on the GPU (different streams or
 *     contexts) race; calls on one stream are ordered. */
int cfr_exploitability_batch_noalloc(cfr_ctx *ctx, double *dev_expl);

/* Exploitability of every game, as cfr_exploitability_batch, written to a
 * caller-owned DEVICE buffer of n_games doubles and left asynchronous on the
 * context's stream (valid once the stream has reached this point: record an
 * event, or call cfr_sync).  The scratch is the context's own, so calls on
 * different contexts and streams may overlap.  A game whose best-response
 * pass gave up on a bounded wait reads as NaN; the status comes with the
 * next synchronising call.  For serving loops that keep many contexts busy
 * without waiting on any one of them. */
int cfr_exploitability_async(cfr_ctx *ctx, double *dev_expl);

/* Copy the state of n games (cumulative regrets, next strategy, average sums
 * and iteration counter; either precision, bit for bit) from context src into
 * context dst, game host_src_games[k] of src into game host_dst_games[k] of
 * dst; the two must be the same game (checked through its sequence,
 * infoset, node and payoff counts).  dst's sequence-form strategies are
 * rebuilt from the copied behavioural ones.  The copy follows the work
 * already issued on src's stream; the call returns once it is complete, so
 * src may be freed right after.  Both contexts must be on one device and
 * have the same precision.  For serving: the unfinished games of a batch are
 * moved, with new requests, into a new context, and the old one's memory is
 * released (the iteration continues exactly as it would have). */
int cfr_copy_game_states(cfr_ctx *dst, int64_t n, const int64_t *host_dst_games, cfr_ctx *src,
                         const int64_t *host_src_games);

/* Checkpoint / resume of game g, player p: cumulative regrets r (S_p), the
 * behavioural strategy to be played next b (S_p), the average sums xbar
 * (S_p + 1, empty sequence first) in FP64, and the completed-iteration count t
 * (shared by both players of a game).  cfr_set_state rebuilds the sequence-form
 * strategy from b on the GPU. */
int cfr_get_state(cfr_ctx *ctx, int64_t game, int player, double *host_r, double *host_b, double *host_xbar,
                  int64_t *t);
int cfr_set_state(cfr_ctx *ctx, int64_t game, int player, const double *host_r, const double *host_b,
                  const double *host_xbar, int64_t t);

/* Intermediate values of game g, player p (1 or 2), FP64, for inspection:
 *   host_x:  S_p + 1 entries, the sequence-form strategy x of Sec. 2.1 that
 *            the player plays next (x[0] = 1 for the empty sequence, then
 *            x[(j,a)] = x[p_j] b_j[a], Alg. 1 NextStrategy), in the caller's
 *            sequence order;
 *   host_ev: J_p entries, ev_j = sum_a b_j[a] V[(j,a)] of each caller infoset
 *            j from this player's last bottom-up pass (Alg. 1 ObserveUtility;
 *            0 before the first iteration or after cfr_set_state).
 * Either pointer may be NULL.  CFR_ERR_STATE unless the context was loaded
 * with the `values` load option. */
int cfr_get_values(cfr_ctx *ctx, int64_t game, int player, double *host_x, double *host_ev);

/* Tracing: run n iterations without CUDA graphs, with a CUDA event recorded
 * between consecutive kernel launches on the context's stream, and return the
 * summed device time (ms) of each launch slot of an iteration in host_ms[4]:
 * [player-1 up, player-1 down, player-2 up, player-2 down] (simultaneous
 * schedule: [p1 up, p2 up, p1 down, p2 down]).  Tracing always launches
 * the two passes of a player separately (load option passes = 2).  The
 * iterations are real: state and counters advance as in cfr_iterate. */
int cfr_profile_iterations(cfr_ctx *ctx, int64_t n, cfr_variant v, double alpha, double beta, double gamma,
                           float *host_ms);

/* Number of kernels the context's iteration calls (cfr_iterate,
 * cfr_iterate_batch, cfr_profile_iterations) have launched so far; each
 * kernel of a replayed CUDA graph counts once per replay. */
int cfr_kernel_launches(cfr_ctx *ctx, int64_t *host_count);

/* Block until all work issued on the context's stream has finished
 * (CFR_ERR_TIMEOUT if a bounded device wait gave up). */
int cfr_sync(cfr_ctx *ctx);

/* Release every resource of the context (NULL is allowed). */
void cfr_free(cfr_ctx *ctx);

/* Static description of a status code. */
const char *cfr_strerror(int status);

/* Message of the last failing call on this host thread ("" if none). */
const char *cfr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CFR_B300_H */
