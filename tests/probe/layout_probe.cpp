// Test-only host wrapper around the game compiler: exposes the compiled layout
// to the CPU tests so its index arrays can be checked without a GPU.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>

#include "../../paper_2605_14277_b300/csrc/layout.h"

using namespace cfrb;

template <class T>
int64_t copy_out(const std::vector<T> &v, void *out) {
    if (out) std::memcpy(out, v.data(), v.size() * sizeof(T));
    return (int64_t)v.size();
}

extern "C" {

void *probe_compile(int64_t G, const int64_t *n, const int32_t *const *parent, const int8_t *const *kind,
                    const int32_t *const *infoset, const int32_t *const *action, const double *const *prob,
                    const double *const *payoff, int64_t item_bytes, char *err, int errlen) {
    std::vector<TreeView> tv(G);
    for (int64_t g = 0; g < G; g++) tv[g] = {n[g], parent[g], kind[g], infoset[g], action[g], prob[g], payoff[g]};
    Layout *L = new Layout();
    CompileOptions o;
    if (const char *f = std::getenv("LAYOUT_PROBE_FLAT")) o.flat = std::atoi(f) != 0;
    if (const char *f = std::getenv("LAYOUT_PROBE_SLOTS")) o.slots = std::atoll(f);
    if (item_bytes > 0) {
        o.item_bytes = item_bytes;
        o.min_item_bytes = std::min<int64_t>(o.min_item_bytes, item_bytes);
    }
    std::string e;
    if (compile_forest(tv.data(), G, o, L, &e) != ST_OK) {
        std::strncpy(err, e.c_str(), errlen - 1);
        delete L;
        return nullptr;
    }
    return L;
}

void probe_free(void *h) { delete (Layout *)h; }

// int32 arrays by name; returns the length (copies when out != NULL)
int64_t probe_i32(void *h, int p, const char *name, void *out) {
    const PlayerLayout &P = ((Layout *)h)->pl[p];
    std::string s(name);
    if (s == "inf_seq") return copy_out(P.inf_seq, out);
    if (s == "seq_child") return copy_out(P.seq_child, out);
    if (s == "inf_par") return copy_out(P.inf_par, out);
    if (s == "seq_game") return copy_out(P.seq_game, out);
    if (s == "m_ptr") return copy_out(P.m_ptr, out);
    if (s == "m_col") return copy_out(P.m_col, out);
    if (s == "ranges") return copy_out(P.ranges, out);
    if (s == "rwin") return copy_out(P.rwin, out);
    if (s == "win") return copy_out(P.win, out);
    if (s == "lcol") return copy_out(P.lcol, out);
    if (s == "up_queue") return copy_out(P.up_queue, out);
    if (s == "down_queue") return copy_out(P.down_queue, out);
    if (s == "game_root") return copy_out(P.game_root, out);
    if (s == "game_tiers") return copy_out(P.game_tiers, out);
    if (s == "danc_off") return copy_out(P.danc_off, out);
    if (s == "ext_inf") return copy_out(P.ext_inf, out);
    if (s == "ext_seq0") return copy_out(P.ext_seq0, out);
    if (s == "units" || s == "dunits") {
        const std::vector<Unit> &v = s == "units" ? P.units : P.dunits;
        if (out)
            for (size_t k = 0; k < v.size(); k++) {
                int32_t *o = (int32_t *)out + 8 * k;
                o[0] = v[k].game; o[1] = v[k].lvl0; o[2] = v[k].nlvl; o[3] = v[k].rng;
                o[4] = v[k].flags; o[5] = v[k].parent; o[6] = v[k].nchild; o[7] = v[k].depth;
            }
        return (int64_t)v.size() * 8;
    }
    return -1;
}

int64_t probe_f64(void *h, int p, const char *name, void *out) {
    const PlayerLayout &P = ((Layout *)h)->pl[p];
    std::string s(name);
    if (s == "m_val64") return copy_out(P.m_val64, out);
    return -1;
}

int64_t probe_i64(void *h, int p, const char *name, void *out) {
    const PlayerLayout &P = ((Layout *)h)->pl[p];
    std::string s(name);
    if (s == "game_jbase") return copy_out(P.game_jbase, out);
    if (s == "game_sbase") return copy_out(P.game_sbase, out);
    return -1;
}

}  // extern "C"
