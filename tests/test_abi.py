"""The C ABI library without a GPU: it loads, exports every function that
include/cfr.h declares, and answers the calls that need no device (shape
table, static error strings, argument checks made before any device work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cfr.h")
HEADER_N = os.path.join(ROOT, "include", "cfr_nplayer.h")
LIB = os.path.join(ROOT, "paper_2605_14277_b300", "libcfr.so")


def declared_functions(header=HEADER, prefix="cfr_"):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)   # drop comments
    names = re.findall(r"^\s*(?:int|int64_t|void|const\s+char\s*\*)\s*\*?\s*(" + prefix + r"\w+)\s*\(", text,
                       flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2605_14277_b300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("cfr_load_tree", "cfr_load_batch", "cfr_iterate", "cfr_get_average_strategy",
                 "cfr_exploitability", "cfr_free", "cfr_strerror", "cfr_load_batch_opts",
                 "cfr_exploitability_batch_noalloc"):
        assert want in names
    assert len(names) >= 20


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_nplayer_header_and_exports(lib):
    names = declared_functions(HEADER_N, "cfrn_")
    for want in ("cfrn_load", "cfrn_iterate", "cfrn_get_state", "cfrn_get_values", "cfrn_nash_conv",
                 "cfrn_get_average_strategy", "cfrn_free", "cfrn_time_passes", "cfrn_launches"):
        assert want in names
    assert [n for n in names if not hasattr(lib, n)] == []


def test_nplayer_calls_that_need_no_device(lib):
    """Invalid trees and arguments are refused before any device work."""
    import numpy as np
    from paper_2605_14277_b300 import games as G
    from paper_2605_14277_b300 import nplayer as NP
    from paper_2605_14277_b300.cfr import CFRError
    NP.lib()
    t = G.kuhn3_game()
    cases = []
    bad = G.kuhn3_game(); bad.parent[5] = 7; cases.append((bad, "parent must precede child at node 5"))
    bad = G.kuhn3_game(); bad.actor[1] = 3; cases.append((bad, "bad actor at node 1"))
    bad = G.kuhn3_game(); bad.kind[3] = 5; cases.append((bad, "bad node kind at node 3"))
    bad = G.kuhn3_game()
    bad.chance_prob[bad.parent == 0] *= 0.5
    cases.append((bad, "chance probabilities do not sum to 1 at node 0"))
    bad = G.kuhn3_game(); bad.action[2] = bad.action[3] if bad.parent[2] == bad.parent[3] else 9
    cases.append((bad, "action index"))
    bad = G.kuhn3_game()
    dec = np.flatnonzero(bad.kind == G.N_DECISION)
    bad.infoset[dec[dec > 30][0]] = 40        # a hole in the ids of that player
    cases.append((bad, "has no node (ids must be dense)"))
    two = G.nplayer_from_two_player(G.small_random_game(1), 2)
    two.n_players = 9
    cases.append((two, "n_players must be 2..8"))
    for tree, msg in cases:
        with pytest.raises(CFRError) as ei:
            NP.NSolver(tree)
        assert ei.value.status == -1 and msg in str(ei.value), str(ei.value)
    # imperfect recall: two nodes of one infoset reached through different own actions
    bad = G.kuhn3_game()
    p0 = np.flatnonzero((bad.kind == G.N_DECISION) & (bad.actor == 0))
    again = p0[bad.parent[p0] != 0][0]          # seat 0 acting a second time (after its own check)
    bad.infoset[again] = bad.infoset[p0[0]]     # merged with a first-action infoset
    with pytest.raises(CFRError) as ei:
        NP.NSolver(bad)
    assert ei.value.status == -1 and "imperfect recall" in str(ei.value)
    assert NP.lib().cfrn_sizes(None, 0, None) == -6
    assert NP.lib().cfrn_iterate(None, 1, 0, 0.0, 0.0, 0.0, 1) == -6
    assert NP.lib().cfrn_set_graph_iterations(None, 4) == -6


def test_calls_that_need_no_device(lib):
    lib.cfr_strerror.restype = ctypes.c_char_p
    assert lib.cfr_strerror(0)
    assert lib.cfr_strerror(-4)
    n = lib.cfr_num_shapes()
    assert n >= 2
    out = (ctypes.c_int32 * 3)()
    for k in range(1, n + 1):
        assert lib.cfr_shape_info(k, out) == 0
        threads, per_sm, buf = out
        assert threads % 32 == 0 and threads >= 128
        assert per_sm >= 1 and buf % 1024 == 0
        # two buffers per CTA fit an SM's shared memory
        assert per_sm * (2 * buf + 8 * 1024) <= 228 * 1024
    assert lib.cfr_shape_info(0, out) == -6
    assert lib.cfr_shape_info(n + 1, out) == -6
    # the shape chosen when none is given: the default for one game of at
    # least 1M nodes, the 256-thread, 3-CTA, 32 KB shape otherwise
    lib.cfr_pick_shape.argtypes = [ctypes.c_int64, ctypes.c_int64]
    d = lib.cfr_default_shape()
    assert lib.cfr_pick_shape(1, 6_000_000) == d
    many = lib.cfr_pick_shape(64, 2_000_000)
    assert lib.cfr_pick_shape(1, 10_000) == many and many != d
    out3 = (ctypes.c_int32 * 3)()
    assert lib.cfr_shape_info(many, out3) == 0 and list(out3) == [256, 3, 32768]
    assert lib.cfr_pick_shape(0, 10) == -6 and lib.cfr_pick_shape(1, 0) == -6


class _Opts(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("flat", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


def test_load_rejects_bad_arguments_before_device_work(lib):
    h = ctypes.c_void_p()
    # no games / NULL output
    assert lib.cfr_load_batch(None, 0, None, ctypes.byref(h)) == -6
    assert lib.cfr_load_batch(None, 1, None, None) == -6
    # bad options are refused before the trees are looked at
    bad = _Opts(99, 0)
    assert lib.cfr_load_batch_opts(None, 1, None, ctypes.byref(bad), ctypes.byref(h)) == -6
    bad = _Opts(0, 2)
    assert lib.cfr_load_batch_opts(None, 1, None, ctypes.byref(bad), ctypes.byref(h)) == -6
    bad = _Opts(0, 0, 3)
    assert lib.cfr_load_batch_opts(None, 1, None, ctypes.byref(bad), ctypes.byref(h)) == -6
    bad = _Opts(0, 0)
    bad.reserved[3] = 1
    assert lib.cfr_load_batch_opts(None, 1, None, ctypes.byref(bad), ctypes.byref(h)) == -6


def test_nplayer_host_compile_matches_the_oracle(lib):
    """The n-player host compiler (no device): every player's infoset,
    sequence and level counts and tensor nonzeros equal the n-player oracle's
    own parse of the same tree; invalid trees give the loader's message."""
    import numpy as np
    from oracle.nplayer import NGame
    from paper_2605_14277_b300 import games as G
    from paper_2605_14277_b300 import nplayer as NP
    from paper_2605_14277_b300.cfr import CFRError
    trees = [G.kuhn3_game(), G.small_nplayer_game(3, 1), G.small_nplayer_game(4, 2),
             G.random_nplayer_game(5, 3, depth=6, chance={0: 2}, actions=(2, 3), zero_sum=False),
             G.random_nplayer_game(8, 4, depth=9, chance={0: 2}, actions=(1, 2), zero_sum=False),
             G.nplayer_from_two_player(G.poker_game(), 3),
             G.nplayer_normal_form([np.arange(12.0).reshape(2, 3, 2) - 5.0] * 3)]
    for tree in trees:
        got = NP.check_tree(tree)
        g = NGame(tree)
        for p, P in enumerate(g.pl):
            nz = int(np.count_nonzero((g.tpay[:, p] != 0.0) & (g.treach != 0.0)))
            want = {"J": P.J, "S": P.S, "levels": len(P.levels), "nnz": nz}
            assert got[p] == want, (tree.name, p, got[p], want)
    bad = G.kuhn3_game()
    bad.parent[5] = 7
    with pytest.raises(CFRError) as ei:
        NP.check_tree(bad)
    assert "parent must precede child at node 5" in str(ei.value)
