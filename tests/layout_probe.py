"""ctypes access to the host game compiler's layout (test-only)."""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2605_14277_b300", "csrc")
SRC = [os.path.join(HERE, "probe", "layout_probe.cpp"), os.path.join(CSRC, "compiler.cpp")]
SO = os.path.join(HERE, "probe", "liblayout_probe.so")

_lib = None


def lib():
    global _lib
    if _lib is None:
        deps = SRC + [os.path.join(CSRC, "layout.h")]
        if not os.path.exists(SO) or any(os.path.getmtime(f) > os.path.getmtime(SO) for f in deps):
            subprocess.check_call(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-pthread", "-o", SO, *SRC])
        L = ctypes.CDLL(SO)
        P = ctypes.c_void_p
        L.probe_compile.restype = P
        L.probe_compile.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, ctypes.c_int64, ctypes.c_char_p,
                                    ctypes.c_int]
        L.probe_free.argtypes = [P]
        for f in (L.probe_i32, L.probe_f64, L.probe_i64):
            f.restype = ctypes.c_int64
            f.argtypes = [P, ctypes.c_int, ctypes.c_char_p, P]
        _lib = L
    return _lib


class Layout:
    def __init__(self, trees, item_bytes=0):
        L = lib()
        G = len(trees)
        self.trees = trees
        keep = []

        def arr(name, dt):
            a = [np.ascontiguousarray(getattr(t, name), dt) for t in trees]
            keep.append(a)
            return (ctypes.c_void_p * G)(*[x.ctypes.data for x in a])

        n = np.array([t.n_nodes for t in trees], dtype=np.int64)
        err = ctypes.create_string_buffer(512)
        h = L.probe_compile(G, n.ctypes.data, arr("parent", np.int32), arr("kind", np.int8),
                            arr("infoset", np.int32), arr("action", np.int32), arr("chance_prob", np.float64),
                            arr("payoff", np.float64), item_bytes, err, 512)
        if not h:
            raise ValueError(err.value.decode())
        self.h = h
        self.pl = {}
        for p in (0, 1):
            d = {}
            for name in ("inf_seq", "seq_child", "inf_par", "seq_game", "m_ptr", "m_col", "ranges", "rwin", "win", "lcol",
                         "up_queue", "down_queue", "game_root", "game_tiers", "ext_inf", "ext_seq0", "units", "dunits",
                         "danc_off"):
                m = L.probe_i32(h, p, name.encode(), None)
                a = np.zeros(m, np.int32)
                L.probe_i32(h, p, name.encode(), a.ctypes.data)
                d[name] = a
            m = L.probe_f64(h, p, b"m_val64", None)
            a = np.zeros(m)
            L.probe_f64(h, p, b"m_val64", a.ctypes.data)
            d["m_val64"] = a
            for name in ("game_jbase", "game_sbase"):
                m = L.probe_i64(h, p, name.encode(), None)
                a = np.zeros(m, np.int64)
                L.probe_i64(h, p, name.encode(), a.ctypes.data)
                d[name] = a
            d["units"] = d["units"].reshape(-1, 8)   # game, lvl0, nlvl, rng, flags, parent, nchild, depth
            d["dunits"] = d["dunits"].reshape(-1, 8)
            self.pl[p] = d

    def __del__(self):
        if getattr(self, "h", None):
            lib().probe_free(self.h)
            self.h = None

    def caller_to_forest(self, p, g):
        """forest sequence index of each caller sequence of game g (player p = 0/1)"""
        d = self.pl[p]
        jb = d["game_jbase"][g]
        J = d["game_jbase"][g + 1] - jb
        S = d["game_sbase"][g + 1] - d["game_sbase"][g]
        out = np.zeros(S, np.int64)
        for k in range(J):
            j = d["ext_inf"][jb + k]
            s0, s1 = d["inf_seq"][j], d["inf_seq"][j + 1]
            base = d["ext_seq0"][jb + k]
            out[base: base + (s1 - s0)] = np.arange(s0, s1)
        return out


def span16(n, e):
    return (n * e + 32 + 15) // 16 * 16


def work16(n, e):
    return (n * e + 15) // 16 * 16


def up_bytes(ns, ni, nz):
    """shared-memory bytes of one staged level of the up pass (layout.h)"""
    return (span16(ns, 8) + span16(ns, 4) + 2 * span16(ns + 1, 4) + span16(ni + 1, 4) + 2 * span16(nz, 4)
            + work16(nz, 4) + work16(ns, 4) + work16(ni, 4))


def down_bytes(ns, ni):
    """shared-memory bytes of one staged level of the down pass (layout.h): b,
    over which the next x is computed in place, infoset parents and segments"""
    return span16(ns, 4) + span16(ni, 4) + span16(ni + 1, 4)
