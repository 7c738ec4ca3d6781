/*
 * cfr_nplayer.h -- C ABI of libcfr.so for n-player games (2 to 8 players):
 * sequence-form CFR whose utility step is a payoff-tensor contraction.
 *
 * "Parallelizing Counterfactual Regret Minimization" (Kim & Sandholm),
 * Sec. 2.1: each player runs sequence-form CFR over its own tree-form
 * sequential decision process, and the utilities it observes come from a
 * sparse matrix-vector product with two players or from tensor operations in
 * multiplayer settings.  Per player i and iteration:
 *
 *   u_i[s] = sum over terminals z with seq_i(z) = s of
 *            pi_c(z) * payoff_i(z) * prod_{k != i} x_k[seq_k(z)]
 *
 * (a sparse tensor with one nonzero per terminal, contracted with the other
 * players' sequence-form strategies), then Alg. 1/2's ObserveUtility and
 * NextStrategy with the post-op of the variant (Alg. 3-5).  Players update in
 * the order 0, 1, ..., n-1 (alternating, Sec. 3.5.1: each sees the strategies
 * the players before it have just recomputed) or all from the iteration's
 * start (simultaneous).  The average strategy is xbar_i += t^gamma x_i^t.
 *
 * Conventions shared with include/cfr.h: status codes (CFR_OK, CFR_ERR_*),
 * variant numbers (CFR_VANILLA .. CFR_PCFR), cfr_strerror.  All calls are
 * synchronous with respect to the host buffers they take (those are copied
 * before the call returns) and asynchronous on the context's stream
 * otherwise; cfrn_sync waits for the stream.
 *
 * Ownership: the context owns every device buffer it allocates; cfrn_free
 * releases them.  The caller owns every host buffer it passes.
 */
#ifndef CFR_NPLAYER_H
#define CFR_NPLAYER_H

#include <stdint.h>

#include "cfr.h"

#ifdef __cplusplus
extern "C" {
#endif

#define CFRN_MAX_PLAYERS 8

/* Node kinds of an n-player tree. */
#define CFRN_CHANCE 0
#define CFRN_DECISION 1
#define CFRN_TERMINAL 2

/* One n-player game tree, nodes in an order where every parent precedes its
 * children (node 0 is the root, parent[0] = -1).
 *   kind[i]        CFRN_CHANCE, CFRN_DECISION or CFRN_TERMINAL
 *   actor[i]       decision nodes: the acting player 0..n_players-1
 *   infoset[i]     decision nodes: infoset id, dense 0..J_p-1 per player; all
 *                  nodes of an infoset have the same number of children and
 *                  the same history of the acting player's own actions
 *                  (perfect recall)
 *   action[i]      non-root nodes: index of the edge from the parent; the
 *                  children of a node carry 0..(children-1), each once
 *   chance_prob[i] children of chance nodes: the edge's probability (they sum
 *                  to 1 per chance node); ignored elsewhere
 *   payoff[i*n+p]  terminals: player p's utility; ignored elsewhere
 * Violations return CFR_ERR_INVALID with a message naming the node
 * (cfrn_last_error). */
typedef struct {
    int64_t n_nodes;
    int32_t n_players;
    const int32_t *parent;
    const int8_t *kind;
    const int8_t *actor;
    const int32_t *infoset;
    const int32_t *action;
    const double *chance_prob;
    const double *payoff;
} cfrn_tree_desc;

typedef struct cfrn_ctx cfrn_ctx;

/* Compile the tree on the host (per-player sequence forms numbered level by
 * level, one payoff-tensor CSR per player) and upload it to the current CUDA
 * device.  stream: a cudaStream_t (not the legacy default stream: iterations
 * are captured as CUDA graphs), or NULL for a stream the context creates and
 * destroys.  The strategies start uniform, regrets and averages at 0, t = 0.
 * Errors: CFR_ERR_INVALID (bad tree), CFR_ERR_CUDA (allocation or copy). */
int cfrn_load(const cfrn_tree_desc *tree, void *stream, cfrn_ctx **out);

/* Compile the tree on the host only (no device work): CFR_OK, or
 * cfrn_load's CFR_ERR_INVALID / CFR_ERR_ARG with the same message.  sizes
 * (may be NULL) receives 4 entries per player: infosets J_p, non-empty
 * sequences S_p, levels of its decision points, nonzeros of its payoff
 * tensor (terminals where its payoff and the chance reach are nonzero). */
int cfrn_check_tree(const cfrn_tree_desc *tree, int64_t *sizes);

/* Release the context (waits for its stream first).  NULL is accepted. */
int cfrn_free(cfrn_ctx *ctx);

/* Message of the last error of this thread (empty if none). */
const char *cfrn_last_error(void);

/* Sizes of player p (CFR_ERR_ARG for a player outside 0..n-1): out[0]
 * infosets J_p, out[1] non-empty sequences S_p, out[2] levels of its decision
 * points, out[3] nonzeros of its payoff tensor, out[4] players, out[5]
 * iterations done, out[6] kernel launches of one iteration (all players). */
int cfrn_sizes(const cfrn_ctx *ctx, int player, int64_t *out);

/* The player's decision points and sequences per level (level 0: the decision
 * points whose parent sequence is the empty one; level l + 1: those below a
 * sequence of level l): out[2l] decision points, out[2l + 1] sequences, for l
 * < min(levels, cap); out (host, 2 * cap entries) belongs to the caller.
 * Errors: CFR_ERR_ARG (bad player, NULL out, cap < 0). */
int cfrn_level_sizes(const cfrn_ctx *ctx, int player, int64_t *out, int cap);

/* Run n iterations of the variant (CFR_VANILLA, CFR_PLUS, CFR_DCFR,
 * CFR_PCFR_PLUS, CFR_PCFR) with DCFR's alpha, beta and the averaging exponent
 * gamma (iteration t adds t^gamma x^t to the average); alternating != 0 for
 * alternating updates.  Iterations run as CUDA graphs of the length set by
 * cfrn_set_graph_iterations (default 64), the rest eagerly.
 * Errors: CFR_ERR_ARG (variant, n < 0), CFR_ERR_CUDA. */
int cfrn_iterate(cfrn_ctx *ctx, int64_t n, int variant, double alpha, double beta, double gamma,
                 int alternating);

/* Iterations per CUDA graph (1..1024; CFR_ERR_ARG otherwise); 1 launches
 * every pass eagerly. */
int cfrn_set_graph_iterations(cfrn_ctx *ctx, int k);

/* Capture (and upload) the CUDA graph cfrn_iterate would use for these
 * arguments, without running it, so that a later timed cfrn_iterate does not
 * pay for the capture.  CFR_ERR_ARG for a bad variant. */
int cfrn_prepare_graph(cfrn_ctx *ctx, int variant, double alpha, double beta, double gamma, int alternating);

/* Wait for the context's stream; CFR_ERR_CUDA if a kernel failed. */
int cfrn_sync(cfrn_ctx *ctx);

/* State of player p in the caller's numbering (infoset ids, then actions):
 * r[S_p] cumulative regrets and b[S_p] the behavioural strategy to be played
 * next (sequence off_j + a, off_j = the actions of infosets 0..j-1), xbar[S_p+1]
 * the average accumulator with the empty sequence first; *t the iterations
 * done.  Any pointer may be NULL.  Waits for the stream. */
int cfrn_get_state(cfrn_ctx *ctx, int player, double *r, double *b, double *xbar, int64_t *t);

/* Resume player p from a checkpoint, in cfrn_get_state's layout: r[S_p],
 * b[S_p] (every infoset's entries >= 0 and summing to 1 within 1e-5, else
 * CFR_ERR_ARG), xbar[S_p+1]; the sequence form x is rebuilt from b.  Any of
 * the three may be NULL (left as it is).  t >= 0 sets the context's iteration
 * counter (shared by the players), t < 0 leaves it.  Waits for the stream. */
int cfrn_set_state(cfrn_ctx *ctx, int player, const double *r, const double *b, const double *xbar, int64_t t);

/* Player p's sequence-form strategy x[S_p+1] (the one it plays next; empty
 * sequence first) and the utility u[S_p+1] that the payoff tensor gives
 * against the other players' current strategies (FP32, computed by the same
 * kernel as an iteration's), in the caller's numbering.  Either pointer may
 * be NULL.  Waits for the stream. */
int cfrn_get_values(cfrn_ctx *ctx, int player, double *x, double *u);

/* Behavioural average strategy of player p: out[S_p] = xbar[(j,a)] / xbar[p_j],
 * uniform where xbar[p_j] = 0 (caller numbering).  Waits for the stream. */
int cfrn_get_average_strategy(cfrn_ctx *ctx, int player, double *out, int64_t len);

/* NashConv of the average profile (each player's xbar / xbar[empty]; the
 * current strategies before any iteration), in FP64 on the device: the sum
 * over players of (best-response value - the player's own value against
 * the others).  gains[n_players] (may be NULL) receives the per-player
 * terms.  Waits for the stream. */
int cfrn_nash_conv(cfrn_ctx *ctx, double *nash_conv, double *gains);

/* Time each kind of pass with CUDA events over `iters` eager iterations (the
 * state advances): us[0] tensor rows with the average update (one kernel),
 * us[1] bottom-up levels, us[2] 0 (no separate kernel), us[3] top-down
 * levels, each the mean per iteration summed over players.  Waits for the
 * stream. */
int cfrn_time_passes(cfrn_ctx *ctx, int iters, int variant, double alpha, double beta, double gamma,
                     int alternating, double *us);

/* Kernel launches the context has issued since it was loaded (graph
 * replays count every kernel they hold). */
int64_t cfrn_launches(const cfrn_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* CFR_NPLAYER_H */
