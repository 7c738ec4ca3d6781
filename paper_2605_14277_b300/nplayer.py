"""Python binding of the n-player entry points of libcfr.so (include/cfr_nplayer.h).

Argument marshalling only: every step of n-player CFR runs in the library's
CUDA kernels.  There is no CPU fallback; without the built library the
binding raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import cfr as _cfr
from .cfr import DEFAULT_PARAMS, VARIANTS, CFRError


class NTreeDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_players", ctypes.c_int32), ("parent", ctypes.c_void_p),
                ("kind", ctypes.c_void_p), ("actor", ctypes.c_void_p), ("infoset", ctypes.c_void_p),
                ("action", ctypes.c_void_p), ("chance_prob", ctypes.c_void_p), ("payoff", ctypes.c_void_p)]


_done = None


def lib():
    global _done
    L = _cfr.lib()
    if _done is not L:
        P, i64, d, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.cfrn_load.argtypes = [ctypes.POINTER(NTreeDesc), P, ctypes.POINTER(P)]
        L.cfrn_free.argtypes = [P]
        L.cfrn_check_tree.argtypes = [ctypes.POINTER(NTreeDesc), P]
        L.cfrn_last_error.argtypes = []
        L.cfrn_last_error.restype = ctypes.c_char_p
        L.cfrn_sizes.argtypes = [P, i, P]
        L.cfrn_level_sizes.argtypes = [P, i, P, i]
        L.cfrn_iterate.argtypes = [P, i64, i, d, d, d, i]
        L.cfrn_set_graph_iterations.argtypes = [P, i]
        L.cfrn_sync.argtypes = [P]
        L.cfrn_prepare_graph.argtypes = [P, i, d, d, d, i]
        L.cfrn_get_state.argtypes = [P, i, P, P, P, P]
        L.cfrn_get_values.argtypes = [P, i, P, P]
        L.cfrn_set_state.argtypes = [P, i, P, P, P, i64]
        L.cfrn_get_average_strategy.argtypes = [P, i, P, i64]
        L.cfrn_nash_conv.argtypes = [P, P, P]
        L.cfrn_time_passes.argtypes = [P, i, i, d, d, d, i, P]
        L.cfrn_launches.argtypes = [P]
        L.cfrn_launches.restype = i64
        _done = L
    return L


def _check(rc: int, where: str):
    if rc != 0:
        raise CFRError(rc, where, lib().cfrn_last_error().decode())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _desc(tree):
    keep = [np.ascontiguousarray(tree.parent, np.int32), np.ascontiguousarray(tree.kind, np.int8),
            np.ascontiguousarray(tree.actor, np.int8), np.ascontiguousarray(tree.infoset, np.int32),
            np.ascontiguousarray(tree.action, np.int32), np.ascontiguousarray(tree.chance_prob, np.float64),
            np.ascontiguousarray(tree.payoff, np.float64).reshape(-1)]
    return NTreeDesc(int(tree.n_nodes), int(tree.n_players), *[a.ctypes.data for a in keep]), keep


def check_tree(tree):
    """Compile the tree on the host only: per player {J, S, levels, nnz}
    (raises CFRError on an invalid tree)."""
    desc, keep = _desc(tree)
    out = np.zeros(4 * max(1, int(tree.n_players)), np.int64)
    _check(lib().cfrn_check_tree(ctypes.byref(desc), _ptr(out)), "cfrn_check_tree")
    return [{"J": int(out[4 * p]), "S": int(out[4 * p + 1]), "levels": int(out[4 * p + 2]), "nnz": int(out[4 * p + 3])}
            for p in range(int(tree.n_players))]


class NSolver:
    """One n-player game on the current CUDA device (include/cfr_nplayer.h)."""

    def __init__(self, tree, stream=None):
        L = lib()
        desc, self._keep = _desc(tree)
        h = ctypes.c_void_p()
        _check(L.cfrn_load(ctypes.byref(desc), _cfr._stream_handle(stream), ctypes.byref(h)), "cfrn_load")
        self._h = h
        self._keep = None
        self.n = int(tree.n_players)
        self.sizes = [self.size(p) for p in range(self.n)]

    def close(self):
        if getattr(self, "_h", None):
            lib().cfrn_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def size(self, p: int) -> dict:
        out = np.zeros(7, np.int64)
        _check(lib().cfrn_sizes(self._h, p, _ptr(out)), "cfrn_sizes")
        return {"J": int(out[0]), "S": int(out[1]), "levels": int(out[2]), "nnz": int(out[3]),
                "players": int(out[4]), "t": int(out[5]), "kernels_per_iteration": int(out[6])}

    def level_sizes(self, p: int):
        """[(decision points, sequences)] of player p's levels, from the top."""
        L = self.sizes[p]["levels"]
        out = np.zeros(2 * max(1, L), np.int64)
        _check(lib().cfrn_level_sizes(self._h, p, _ptr(out), L), "cfrn_level_sizes")
        return [(int(out[2 * l]), int(out[2 * l + 1])) for l in range(L)]

    @property
    def t(self) -> int:
        return self.size(0)["t"]

    def set_graph_iterations(self, k: int):
        _check(lib().cfrn_set_graph_iterations(self._h, int(k)), "cfrn_set_graph_iterations")

    def iterate(self, n: int, variant="dcfr", alpha=None, beta=None, gamma=None, alternating=True):
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        a0, b0, g0 = DEFAULT_PARAMS[v]
        a = a0 if alpha is None else alpha
        b = b0 if beta is None else beta
        g = g0 if gamma is None else gamma
        _check(lib().cfrn_iterate(self._h, int(n), v, float(a), float(b), float(g), int(bool(alternating))),
               "cfrn_iterate")

    def prepare_graph(self, variant="dcfr", alpha=None, beta=None, gamma=None, alternating=True):
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        a0, b0, g0 = DEFAULT_PARAMS[v]
        _check(lib().cfrn_prepare_graph(self._h, v, float(a0 if alpha is None else alpha),
                                        float(b0 if beta is None else beta), float(g0 if gamma is None else gamma),
                                        int(bool(alternating))), "cfrn_prepare_graph")

    def sync(self):
        _check(lib().cfrn_sync(self._h), "cfrn_sync")

    def get_state(self, p: int) -> dict:
        S = self.sizes[p]["S"]
        r, b, xb = np.zeros(S), np.zeros(S), np.zeros(S + 1)
        t = ctypes.c_int64()
        _check(lib().cfrn_get_state(self._h, p, _ptr(r), _ptr(b), _ptr(xb), ctypes.byref(t)), "cfrn_get_state")
        return {"r": r, "b": b, "xbar": xb, "t": t.value}

    def set_state(self, p: int, r=None, b=None, xbar=None, t: int = -1):
        S = self.sizes[p]["S"]

        def arr(a, n):
            if a is None:
                return None
            a = np.ascontiguousarray(a, np.float64)
            if a.shape != (n,):
                raise ValueError(f"expected {n} entries, got {a.shape}")
            return a
        r, b, xbar = arr(r, S), arr(b, S), arr(xbar, S + 1)
        _check(lib().cfrn_set_state(self._h, p, _ptr(r), _ptr(b), _ptr(xbar), int(t)), "cfrn_set_state")

    def get_values(self, p: int):
        S = self.sizes[p]["S"]
        x, u = np.zeros(S + 1), np.zeros(S + 1)
        _check(lib().cfrn_get_values(self._h, p, _ptr(x), _ptr(u)), "cfrn_get_values")
        return x, u

    def average_strategy(self, p: int):
        S = self.sizes[p]["S"]
        out = np.zeros(S)
        _check(lib().cfrn_get_average_strategy(self._h, p, _ptr(out), S), "cfrn_get_average_strategy")
        return out

    def nash_conv(self):
        g = np.zeros(self.n)
        v = ctypes.c_double()
        _check(lib().cfrn_nash_conv(self._h, ctypes.byref(v), _ptr(g)), "cfrn_nash_conv")
        return v.value, g

    def time_passes(self, iters: int, variant="dcfr", alpha=None, beta=None, gamma=None, alternating=True):
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        a0, b0, g0 = DEFAULT_PARAMS[v]
        us = np.zeros(4)
        _check(lib().cfrn_time_passes(self._h, int(iters), v, float(a0 if alpha is None else alpha),
                                      float(b0 if beta is None else beta), float(g0 if gamma is None else gamma),
                                      int(bool(alternating)), _ptr(us)), "cfrn_time_passes")
        return {"rows": us[0], "up": us[1], "down": us[3]}

    @property
    def launches(self) -> int:
        return int(lib().cfrn_launches(self._h))
