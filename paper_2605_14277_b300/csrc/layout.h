// Host-side layout of a forest of games for the CUDA passes.
//
// Every per-player vector follows one numbering, a breadth-first order over
// the forest of all loaded games: level 0 holds one pseudo-infoset per game
// (the root, whose single sequence is the empty sequence of that game), level
// d holds the infosets whose parent sequence is at level d-1, sorted by parent
// sequence.  Sequences are numbered in infoset order.  With that order:
//   * the sequences of infoset j are [inf_seq[j], inf_seq[j+1])            (logic matrix C, Sec. 3.1)
//   * the child infosets of sequence s are [seq_child[s], seq_child[s+1])  (level graphs L^(d), Sec. 3.2)
//   * within one level, each game's infosets are contiguous, and so are the
//     descendants of any contiguous range: a unit of work is one contiguous
//     range per level.
#pragma once
#include <cstdint>
#ifndef __CUDACC__
#define __host__
#define __device__
#endif
#include <string>
#include <vector>

namespace cfrb {

struct TreeView {
    int64_t n_nodes;
    const int32_t *parent;
    const int8_t *kind;
    const int32_t *infoset;
    const int32_t *action;
    const double *chance_prob;
    const double *payoff;
};

// One unit of work: levels [lvl0, lvl0 + nlvl) of one game below one
// contiguous range of infosets at level lvl0.  Level k of the unit is
// described by kLvl ints at ranges[rng + kLvl * k]:
//   infosets [j0, j1), sequences [s0, s1), payoff nonzeros [n0, n1)
// (rows s0..s1 of this player's payoff CSR), so a kernel can issue every copy
// of the unit without first reading index arrays.
//
// The units of a game form a tree.  A unit's parent is the unit whose deepest
// level holds the parent sequences of this unit's top-level infosets; the
// game's root unit starts at level 0.  A unit with children ("internal") finds
// the child infosets of its deepest level at the top levels of its child
// units.  Bottom-up passes take every leaf, then the internal units deepest
// first, from one queue; an internal unit stages its own arrays at once and
// starts computing when all its children are done.  The top-down pass works
// units of its own (dunits below): runs of sibling units, each carrying its
// ancestor chain, so that no top-down unit depends on another.
constexpr int kLvl = 6;
struct Unit {
    int32_t game, lvl0, nlvl, rng;
    int32_t flags;    // kStaged | kInternal
    int32_t parent;   // -1: the game's root unit
    int32_t nchild;   // child units
    int32_t depth;    // in the unit tree (root = 0)
};
constexpr int kStaged = 1;       // the unit fits one shared-memory buffer in both passes
constexpr int kInternal = 2;     // the deepest level's child infosets are other units' top levels;
                                 // their range [c0, c1) follows the unit's levels as one more
                                 // kLvl record {c0, c1, 0, 0, 0, 0}
constexpr int kChildOfRoot = 4;  // the parent is the game's root unit (informational)
constexpr int kAncShift = 16;    // top-down units: flags >> kAncShift = levels of the ancestor chain
                                 // staged before the unit's own levels (computed, not written back)
constexpr int kMaxStagedLevels = 24;
constexpr int32_t kWinGap = 16;   // x windows: columns further apart than this start a new window
constexpr int64_t kMaxWin = 32;   // x windows: at most this many per staged level

// Shared-memory bytes a staged unit level needs (host and device agree on
// these): copied ranges get 32 bytes of slack for 16-byte alignment.
__host__ __device__ inline int64_t span16(int64_t n, int e) { return (n * e + 32 + 15) / 16 * 16; }
__host__ __device__ inline int64_t work16(int64_t n, int e) { return (n * e + 15) / 16 * 16; }
// xb: bytes of the level's x area (the other player's x, per payoff entry
// when gathered, or as copied windows of it)
__host__ __device__ inline int64_t up_level_bytes_x(int64_t ns, int64_t ni, int64_t nz, int64_t xb) {
    // r (float2), b, seq_child, payoff row pointers, infoset segments, payoff
    // columns, payoff values; work: the x area, V per sequence, ev per infoset
    return span16(ns, 8) + span16(ns, 4) + 2 * span16(ns + 1, 4) + span16(ni + 1, 4) + 2 * span16(nz, 4) + xb +
           work16(ns, 4) + work16(ni, 4);
}
__host__ __device__ inline int64_t up_level_bytes(int64_t ns, int64_t ni, int64_t nz) {
    return up_level_bytes_x(ns, ni, nz, work16(nz, 4));
}
__host__ __device__ inline int64_t down_level_bytes(int64_t ns, int64_t ni) {
    // b (the next x is computed in place over it), infoset parents, infoset segments
    return span16(ns, 4) + span16(ni, 4) + span16(ni + 1, 4);
}

struct PlayerLayout {
    int64_t S = 0, J = 0;               // forest totals (including the G empty sequences / roots)
    int32_t n_levels = 0;
    std::vector<int32_t> inf_seq;       // [J + 1]
    std::vector<int32_t> seq_child;     // [S + 1]
    std::vector<int32_t> inf_par;       // [J]   parent sequence, -1 for roots
    std::vector<int32_t> seq_game;      // [S]
    std::vector<int32_t> m_ptr;         // [S + 1] payoff rows indexed by this player's sequence
    std::vector<int32_t> m_col;         // [Z]     other player's sequence
    std::vector<float> m_val;           // [Z]     sum over terminals of chance reach * u1
    std::vector<double> m_val64;        // [Z]
    std::vector<Unit> units;            // every unit of every game
    std::vector<int32_t> ranges;        // kLvl ints per level of every unit
    // The other player's x as seen by one staged level's payoff entries: either
    // gathered per entry, or (when the entries' columns cluster) copied in as
    // a few contiguous windows [c0, c1) of it, placed one after another in
    // the level's x area (each span16 bytes, its first column c0 % 4 floats
    // in).  rwin holds {w0, w1, x-area bytes, 0} per range record (in `ranges`
    // order); a staged unit's windows are the contiguous run win[w0 of its
    // first level .. w1 of its last), 4 ints each: {c0, c1, byte offset in
    // the level's x area, level within the unit}; w0 == w1 means gathered.
    // lcol is the staged column array: for a windowed level, the entry's
    // float index into its level's x area; otherwise m_col.
    std::vector<int32_t> rwin;          // 4 ints per range record
    std::vector<int32_t> win;           // 4 ints per window
    std::vector<int32_t> lcol;          // [Z]
    std::vector<int32_t> up_queue;      // leaves largest first, then internal units deepest first
    std::vector<Unit> dunits;           // top-down units: runs of sibling units merged up to the
                                        // smallest footprint cap (within the buffer) that leaves no
                                        // more units than CTAs resident at once, so the pass is one
                                        // round; parent / nchild / depth in this tree.  Their
                                        // range records start with the ancestor chain (flags >>
                                        // kAncShift levels, from level 0 down), then their own levels
    std::vector<int32_t> danc_off;      // [dunits] offset of the unit's ancestors' x in the scratch
                                        // area that units worked from global memory use (xanc_size)
    int64_t xanc_size = 0;
    std::vector<int32_t> down_queue;    // all top-down units by tree depth, then largest first
    std::vector<int32_t> game_root;     // [G] root unit of each game
    std::vector<int32_t> game_tiers;    // [G] depth of the game's unit tree + 1
    // caller order: game g's caller infoset k is ext_inf[game_jbase[g] + k]; its
    // sequences start at caller index ext_seq0[game_jbase[g] + k]
    std::vector<int32_t> ext_inf, ext_seq0;
    std::vector<int64_t> game_jbase, game_sbase;   // caller-order prefix sums over games
    std::vector<int32_t> game_J, game_S;           // caller counts per game
    int32_t max_actions = 0;
};

struct Layout {
    int64_t G = 0, Z = 0;
    PlayerLayout pl[2];
    std::vector<int64_t> game_nodes;
    std::vector<int64_t> game_nnz;
    std::vector<double> game_range;     // max u1 - min u1 over terminals
};

struct CompileOptions {
    int64_t item_bytes = 48 * 1024;    // shared-memory buffer of one staged unit
    int64_t min_item_bytes = 8 * 1024; // smallest unit the packer aims for
    int64_t slots = 296;               // CTAs resident at once (units are sized to give each ~2)
    int64_t internal_div = 2;          // internal units aim for target / internal_div (smaller
                                       // units shorten the chain above the leaves)
    int leaf_order = 0;                // 0: largest first; 1: tree order (children of one parent together)
    bool flat = false;                 // one level per unit below a root unit that holds the narrow top
};

// status codes shared with the C ABI
enum { ST_OK = 0, ST_INVALID = -1, ST_OOM = -2 };

int compile_forest(const TreeView *games, int64_t n_games, const CompileOptions &opt, Layout *out,
                   std::string *err);

}  // namespace cfrb
