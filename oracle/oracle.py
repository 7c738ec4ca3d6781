"""ctypes front-end of the plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product library never does.  The C
source (``cfr_oracle.c``) follows Alg. 1 and the CFR+/DCFR/PCFR+ excerpts
(Alg. 3-5) step by step in FP64; see its header for the passage behind each
step.

All per-sequence vectors are in the caller's (infoset id, action) order:
``r`` and ``b`` have S_i entries, ``xbar`` and sequence-form strategies have
S_i + 1 entries with the empty sequence first.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cfr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

VARIANTS = {"cfr": 0, "cfr+": 1, "dcfr": 2, "pcfr+": 3, "pcfr": 4}
# per-variant defaults: (alternating, alpha, beta, gamma)
DEFAULTS = {0: (False, 0.0, 0.0, 0.0), 1: (True, 0.0, 0.0, 1.0),
            2: (True, 1.5, 0.0, 2.0), 3: (True, 0.0, 0.0, 2.0), 4: (True, 0.0, 0.0, 0.0)}


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        d = ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_build.argtypes = [i64, P, P, P, P, P, P, ctypes.POINTER(P)]
        L.oracle_free.argtypes = [P]
        L.oracle_free.restype = None
        L.oracle_sizes.argtypes = [P, P]
        L.oracle_iterate.argtypes = [P, i64, ctypes.c_int, d, d, d, ctypes.c_int]
        L.oracle_exploitability.argtypes = [P, dp, dp, dp]
        L.oracle_exploitability_of.argtypes = [P, P, P, dp, dp, dp]
        L.oracle_get_state.argtypes = [P, ctypes.c_int, P, P, P, ctypes.POINTER(i64)]
        L.oracle_set_state.argtypes = [P, ctypes.c_int, P, P, P, i64]
        L.oracle_average_strategy.argtypes = [P, ctypes.c_int, P]
        L.oracle_regret_matching.argtypes = [P, ctypes.c_int, P, P]
        L.oracle_sequence_form.argtypes = [P, ctypes.c_int, P, P]
        L.oracle_utility.argtypes = [P, ctypes.c_int, P, P]
        L.oracle_observe_utility.argtypes = [P, ctypes.c_int, P, P, P, P, P]
        L.oracle_infosets.argtypes = [P, ctypes.c_int, P, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.shape[0] != n:
        raise ValueError(f"expected length {n}, got {a.shape[0]}")
    return a


class OracleError(RuntimeError):
    pass


class Oracle:
    """One game in the oracle.  ``Oracle(tree)`` compiles the tree."""

    def __init__(self, tree):
        L = lib()
        self._keep = (tree.parent, tree.kind, tree.infoset, tree.action, tree.chance_prob,
                      tree.payoff)
        h = ctypes.c_void_p()
        rc = L.oracle_build(tree.n_nodes, _ptr(tree.parent), _ptr(tree.kind), _ptr(tree.infoset),
                            _ptr(tree.action), _ptr(tree.chance_prob), _ptr(tree.payoff),
                            ctypes.byref(h))
        if rc != 0:
            raise OracleError(f"oracle_build failed ({rc})")
        self._h = h
        s = np.zeros(6, dtype=np.int64)
        L.oracle_sizes(h, _ptr(s))
        self.S = {1: int(s[0]), 2: int(s[1])}
        self.J = {1: int(s[2]), 2: int(s[3])}
        self.n_terminals = int(s[4])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_free(h)
            self._h = None

    @property
    def t(self) -> int:
        s = np.zeros(6, dtype=np.int64)
        lib().oracle_sizes(self._h, _ptr(s))
        return int(s[5])

    def iterate(self, n: int, variant="cfr", alpha=None, beta=None, gamma=None, alternating=None):
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        alt0, a0, b0, g0 = DEFAULTS[v]
        alpha = a0 if alpha is None else alpha
        beta = b0 if beta is None else beta
        gamma = g0 if gamma is None else gamma
        alternating = alt0 if alternating is None else alternating
        rc = lib().oracle_iterate(self._h, int(n), v, float(alpha), float(beta), float(gamma),
                                  int(bool(alternating)))
        if rc != 0:
            raise OracleError(f"oracle_iterate failed ({rc})")

    def exploitability(self):
        e, b1, b2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lib().oracle_exploitability(self._h, ctypes.byref(e), ctypes.byref(b1), ctypes.byref(b2))
        return e.value, b1.value, b2.value

    def exploitability_of(self, x, y):
        x = _f64(x, self.S[1] + 1)
        y = _f64(y, self.S[2] + 1)
        e, b1, b2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lib().oracle_exploitability_of(self._h, _ptr(x), _ptr(y), ctypes.byref(e),
                                       ctypes.byref(b1), ctypes.byref(b2))
        return e.value, b1.value, b2.value

    def get_state(self, p: int):
        S = self.S[p]
        r, b, xb = np.zeros(S), np.zeros(S), np.zeros(S + 1)
        t = ctypes.c_int64()
        lib().oracle_get_state(self._h, p, _ptr(r), _ptr(b), _ptr(xb), ctypes.byref(t))
        return {"r": r, "b": b, "xbar": xb, "t": t.value}

    def set_state(self, p: int, r, b, xbar, t: int):
        S = self.S[p]
        r, b, xbar = _f64(r, S), _f64(b, S), _f64(xbar, S + 1)
        rc = lib().oracle_set_state(self._h, p, _ptr(r), _ptr(b), _ptr(xbar), int(t))
        if rc != 0:
            raise OracleError(f"oracle_set_state failed ({rc})")

    def average_strategy(self, p: int):
        out = np.zeros(self.S[p])
        lib().oracle_average_strategy(self._h, p, _ptr(out))
        return out

    def regret_matching(self, p: int, r):
        r = _f64(r, self.S[p])
        b = np.zeros(self.S[p])
        lib().oracle_regret_matching(self._h, p, _ptr(r), _ptr(b))
        return b

    def sequence_form(self, p: int, b):
        b = _f64(b, self.S[p])
        x = np.zeros(self.S[p] + 1)
        lib().oracle_sequence_form(self._h, p, _ptr(b), _ptr(x))
        return x

    def utility(self, p: int, xo):
        q = 2 if p == 1 else 1
        xo = _f64(xo, self.S[q] + 1)
        u = np.zeros(self.S[p] + 1)
        lib().oracle_utility(self._h, p, _ptr(xo), _ptr(u))
        return u

    def observe_utility(self, p: int, u, b, r):
        """ObserveUtility with explicit inputs; returns (r_new, V, ev)."""
        u = _f64(u, self.S[p] + 1)
        b = _f64(b, self.S[p])
        r = _f64(r, self.S[p]).copy()
        V = np.zeros(self.S[p] + 1)
        ev = np.zeros(max(self.J[p], 1))
        lib().oracle_observe_utility(self._h, p, _ptr(u), _ptr(b), _ptr(r), _ptr(V), _ptr(ev))
        return r, V, ev[: self.J[p]]

    def infosets(self, p: int):
        """(parent sequence in caller numbering, -1 = empty; action count) per infoset."""
        J = self.J[p]
        ps = np.zeros(max(J, 1), dtype=np.int64)
        na = np.zeros(max(J, 1), dtype=np.int32)
        lib().oracle_infosets(self._h, p, _ptr(ps), _ptr(na))
        return ps[:J], na[:J]
