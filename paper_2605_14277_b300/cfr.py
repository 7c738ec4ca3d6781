"""Python binding of libcfr.so (argument marshalling only).

Every step of CFR runs in the library's CUDA kernels; this module converts
numpy arrays and torch stream handles into the C ABI of ``include/cfr.h`` and
back.  Importing it on a machine without the built library raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcfr.so")

VARIANTS = {"cfr": 0, "vanilla": 0, "cfr+": 1, "dcfr": 2, "pcfr+": 3, "pcfr": 4}
# default (alpha, beta, gamma) per variant: DCFR (1.5, 0) with quadratic
# averaging; CFR+ linear averaging; PCFR+ quadratic; vanilla uniform
DEFAULT_PARAMS = {0: (0.0, 0.0, 0.0), 1: (0.0, 0.0, 1.0), 2: (1.5, 0.0, 2.0), 3: (0.0, 0.0, 2.0), 4: (0.0, 0.0, 0.0)}
UPDATES = {"default": 0, "simultaneous": 1, "alternating": 2}


class CFRError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class LoadOptions(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("flat", ctypes.c_int32), ("passes", ctypes.c_int32),
                ("values", ctypes.c_int32), ("wait_us", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class TreeDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("parent", ctypes.c_void_p), ("kind", ctypes.c_void_p),
                ("infoset", ctypes.c_void_p), ("action", ctypes.c_void_p),
                ("chance_prob", ctypes.c_void_p), ("payoff_p1", ctypes.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcfr.so is not built ({LIB_PATH}); run python -m paper_2605_14277_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, d, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.cfr_load_tree.argtypes = [ctypes.POINTER(TreeDesc), P, ctypes.POINTER(P)]
        L.cfr_load_batch.argtypes = [ctypes.POINTER(TreeDesc), i64, P, ctypes.POINTER(P)]
        L.cfr_load_batch_opts.argtypes = [ctypes.POINTER(TreeDesc), i64, P, ctypes.POINTER(LoadOptions),
                                          ctypes.POINTER(P)]
        L.cfr_num_shapes.argtypes = []
        L.cfr_default_shape.argtypes = []
        L.cfr_pick_shape.argtypes = [ctypes.c_int64, ctypes.c_int64]
        L.cfr_shape_info.argtypes = [i, P]
        L.cfr_iterate.argtypes = [P, i64, i, d, d, d]
        L.cfr_iterate_batch.argtypes = [P, i64, i, d, d, d, P]
        L.cfr_set_update_mode.argtypes = [P, i]
        L.cfr_set_graph_iterations.argtypes = [P, i]
        L.cfr_prepare_graph.argtypes = [P, i, d, d, d]
        L.cfr_sizes.argtypes = [P, i64, P]
        L.cfr_get_average_strategy.argtypes = [P, i64, i, P, i64]
        L.cfr_exploitability.argtypes = [P, P, P, P]
        L.cfr_exploitability_batch.argtypes = [P, P, P, P]
        L.cfr_get_state.argtypes = [P, i64, i, P, P, P, P]
        L.cfr_set_state.argtypes = [P, i64, i, P, P, P, i64]
        L.cfr_get_values.argtypes = [P, i64, i, P, P]
        L.cfr_profile_iterations.argtypes = [P, i64, i, d, d, d, P]
        L.cfr_exploitability_batch_noalloc.argtypes = [P, P]
        L.cfr_exploitability_async.argtypes = [P, P]
        L.cfr_copy_game_states.argtypes = [P, i64, P, P, P]
        L.cfr_sync.argtypes = [P]
        L.cfr_kernel_launches.argtypes = [P, P]
        L.cfr_free.argtypes = [P]
        L.cfr_free.restype = None
        L.cfr_strerror.argtypes = [i]
        L.cfr_strerror.restype = ctypes.c_char_p
        L.cfr_last_error.argtypes = []
        L.cfr_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def default_shape() -> int:
    """The launch shape the library uses for a single large game when none is chosen."""
    return int(lib().cfr_default_shape())


def pick_shape(n_games: int, total_nodes: int) -> int:
    """The launch shape the library uses, when none is chosen, for a load of
    n_games games of total_nodes nodes in all."""
    k = int(lib().cfr_pick_shape(int(n_games), int(total_nodes)))
    _check(min(k, 0), "cfr_pick_shape")
    return k


def shapes():
    """Launch shapes: {k: (threads per CTA, CTAs per SM, unit buffer bytes)}."""
    L = lib()
    out = {}
    for k in range(1, L.cfr_num_shapes() + 1):
        v = np.zeros(3, dtype=np.int32)
        _check(L.cfr_shape_info(k, _ptr(v)), "cfr_shape_info")
        out[k] = tuple(int(x) for x in v)
    return out


def _check(rc: int, where: str):
    if rc != 0:
        L = lib()
        raise CFRError(rc, where, (L.cfr_last_error() or L.cfr_strerror(rc)).decode())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)   # torch.cuda.Stream


def _desc(tree, keep):
    arrs = (np.ascontiguousarray(tree.parent, np.int32), np.ascontiguousarray(tree.kind, np.int8),
            np.ascontiguousarray(tree.infoset, np.int32), np.ascontiguousarray(tree.action, np.int32),
            np.ascontiguousarray(tree.chance_prob, np.float64), np.ascontiguousarray(tree.payoff, np.float64))
    keep.append(arrs)
    return TreeDesc(arrs[0].shape[0], *[a.ctypes.data for a in arrs])


def _resolve(variant, alpha, beta, gamma):
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    a0, b0, g0 = DEFAULT_PARAMS[v]
    return v, (a0 if alpha is None else alpha), (b0 if beta is None else beta), (g0 if gamma is None else gamma)


class _Round:
    """A round queued by Solver.start_round."""

    def __init__(self, solver, event):
        self._s, self._ev = solver, event

    def done(self) -> bool:
        return bool(self._ev.query())

    def result(self):
        self._ev.synchronize()
        self._s.sync()   # a bounded device wait that gave up is reported here
        return self._s._host_expl.numpy().copy()


class Solver:
    """CFR state of one game or of a batch of games resident on the GPU.

    ``Solver(tree)`` loads one game; ``Solver([t1, t2, ...])`` loads a batch
    advanced together by every launch.  ``shape``, ``flat`` and ``passes`` are
    the load options of the C ABI (launch shape, unit layout, one or two
    launches per player and half-iteration; 0 / False = the library's
    choice); every choice computes the same iterations.  ``values`` keeps every
    infoset's counterfactual value for ``get_values``; ``wait_us`` bounds a
    unit's wait for the units it depends on (0 = the library's 1 s);
    ``precision`` 64 runs every pass in FP64 (default 32: FP32 passes)."""

    def __init__(self, trees, stream=None, shape: int = 0, flat: bool = False, passes: int = 0,
                 values: bool = False, wait_us: int = 0, precision: int = 32):
        L = lib()
        batch = isinstance(trees, (list, tuple))
        trees = list(trees) if batch else [trees]
        keep = []
        descs = (TreeDesc * len(trees))(*[_desc(t, keep) for t in trees])
        h = ctypes.c_void_p()
        opts = LoadOptions(int(shape), int(bool(flat)), int(passes), int(bool(values)), int(wait_us), int(precision))
        _check(L.cfr_load_batch_opts(descs, len(trees), _stream_handle(stream), ctypes.byref(opts), ctypes.byref(h)),
               "cfr_load_batch_opts")
        self.shape, self.flat, self.passes = int(shape), bool(flat), int(passes)
        self._torch_stream = stream if (stream is not None and not isinstance(stream, int)) else None
        self._dev_expl = self._host_expl = None
        self._h = h
        self.n_games = len(trees)
        self.batch = batch
        self._sizes = {}   # per game, read on first use (each read waits for the stream)

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.cfr_free(self._h)
            self._h = None

    __del__ = close

    def _game_sizes(self, game: int) -> dict:
        if game not in self._sizes:
            self._sizes[game] = self.sizes(game)
        return self._sizes[game]

    def sizes(self, game: int = 0) -> dict:
        out = np.zeros(10, dtype=np.int64)
        _check(lib().cfr_sizes(self._h, game, _ptr(out)), "cfr_sizes")
        return {"S1": int(out[0]), "S2": int(out[1]), "J1": int(out[2]), "J2": int(out[3]),
                "nnz": int(out[4]), "nodes": int(out[5]), "t": int(out[6]), "games": int(out[7]),
                "device_bytes": int(out[8]), "h2d_bytes": int(out[9])}

    def set_update_mode(self, mode: str):
        _check(lib().cfr_set_update_mode(self._h, UPDATES[mode]), "cfr_set_update_mode")

    def set_graph_iterations(self, k: int):
        _check(lib().cfr_set_graph_iterations(self._h, int(k)), "cfr_set_graph_iterations")

    def prepare_graph(self, variant="cfr", alpha=None, beta=None, gamma=None):
        """Capture now the CUDA graph iterate() will replay (nothing runs)."""
        v, a, b, g = _resolve(variant, alpha, beta, gamma)
        _check(lib().cfr_prepare_graph(self._h, v, a, b, g), "cfr_prepare_graph")

    def iterate(self, n: int, variant="cfr", alpha=None, beta=None, gamma=None, active=None):
        v, a, b, g = _resolve(variant, alpha, beta, gamma)
        if active is None:
            _check(lib().cfr_iterate(self._h, int(n), v, a, b, g), "cfr_iterate")
        else:
            act = np.ascontiguousarray(active, dtype=np.uint8)
            if act.shape[0] != self.n_games:
                raise ValueError("active mask length must equal the number of games")
            _check(lib().cfr_iterate_batch(self._h, int(n), v, a, b, g, _ptr(act)), "cfr_iterate_batch")

    def profile(self, n: int, variant="cfr", alpha=None, beta=None, gamma=None):
        """Summed device ms of the four launch slots over n eager iterations."""
        v, a, b, g = _resolve(variant, alpha, beta, gamma)
        ms = np.zeros(4, dtype=np.float32)
        _check(lib().cfr_profile_iterations(self._h, int(n), v, a, b, g, _ptr(ms)), "cfr_profile_iterations")
        return ms.astype(np.float64)

    def sync(self):
        _check(lib().cfr_sync(self._h), "cfr_sync")

    def kernel_launches(self) -> int:
        """Kernels launched so far by this solver's iteration calls."""
        n = ctypes.c_int64()
        _check(lib().cfr_kernel_launches(self._h, ctypes.byref(n)), "cfr_kernel_launches")
        return int(n.value)

    def exploitability(self):
        e, b1, b2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().cfr_exploitability(self._h, ctypes.byref(e), ctypes.byref(b1), ctypes.byref(b2)),
               "cfr_exploitability")
        return e.value, b1.value, b2.value

    def exploitability_batch(self):
        e, b1, b2 = (np.zeros(self.n_games) for _ in range(3))
        _check(lib().cfr_exploitability_batch(self._h, _ptr(e), _ptr(b1), _ptr(b2)), "cfr_exploitability_batch")
        return e, b1, b2

    def exploitability_into(self, dev_ptr: int):
        """Exploitability of every game written to a caller-owned device buffer
        of n_games doubles (a device address, e.g. torch's tensor.data_ptr()),
        without any allocation; asynchronous on the solver's stream."""
        _check(lib().cfr_exploitability_batch_noalloc(self._h, ctypes.c_void_p(int(dev_ptr))),
               "cfr_exploitability_batch_noalloc")

    def exploitability_async(self, dev_ptr: int):
        """Exploitability of every game into a caller-owned device buffer of
        n_games doubles (a device address), asynchronous on the solver's
        stream; the solver's own scratch, so solvers may overlap."""
        _check(lib().cfr_exploitability_async(self._h, ctypes.c_void_p(int(dev_ptr))), "cfr_exploitability_async")

    def start_round(self, n: int, variant="cfr", active=None, alpha=None, beta=None, gamma=None):
        """n iterations, then the exploitability of every game, all queued on
        the solver's stream without waiting; returns a handle whose done()
        polls and whose result() returns the exploitabilities (and reports a
        device timeout).  Needs a torch stream at construction."""
        import torch
        if self._torch_stream is None:
            raise ValueError("start_round needs Solver(..., stream=torch.cuda.Stream())")
        if self._dev_expl is None:
            self._dev_expl = torch.empty(self.n_games, dtype=torch.float64, device=self._torch_stream.device)
            self._host_expl = torch.empty(self.n_games, dtype=torch.float64, pin_memory=True)
        self.iterate(n, variant, alpha=alpha, beta=beta, gamma=gamma, active=active)
        self.exploitability_async(self._dev_expl.data_ptr())
        with torch.cuda.stream(self._torch_stream):
            self._host_expl.copy_(self._dev_expl, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self._torch_stream)
        return _Round(self, ev)

    def copy_states_from(self, src: "Solver", dst_games, src_games):
        """Take the state of games src_games of `src` (same games) into games
        dst_games of this solver, exactly; returns once the copy is done."""
        d = np.ascontiguousarray(dst_games, dtype=np.int64)
        s_ = np.ascontiguousarray(src_games, dtype=np.int64)
        if d.shape != s_.shape:
            raise ValueError("game lists must have the same length")
        _check(lib().cfr_copy_game_states(self._h, d.shape[0], _ptr(d), src._h, _ptr(s_)), "cfr_copy_game_states")

    def average_strategy(self, player: int, game: int = 0):
        S = self._game_sizes(game)["S1" if player == 1 else "S2"]
        out = np.zeros(S)
        _check(lib().cfr_get_average_strategy(self._h, game, player, _ptr(out), S), "cfr_get_average_strategy")
        return out

    def get_state(self, player: int, game: int = 0):
        S = self._game_sizes(game)["S1" if player == 1 else "S2"]
        r, b, xb = np.zeros(S), np.zeros(S), np.zeros(S + 1)
        t = ctypes.c_int64()
        _check(lib().cfr_get_state(self._h, game, player, _ptr(r), _ptr(b), _ptr(xb), ctypes.byref(t)),
               "cfr_get_state")
        return {"r": r, "b": b, "xbar": xb, "t": t.value}

    def get_values(self, player: int, game: int = 0):
        """The sequence-form strategy to be played next (S + 1 entries, empty
        sequence first) and each infoset's ev from the player's last bottom-up
        pass (J entries), caller order; needs ``Solver(..., values=True)``."""
        sz = self._game_sizes(game)
        S, J = sz["S1" if player == 1 else "S2"], sz["J1" if player == 1 else "J2"]
        x, ev = np.zeros(S + 1), np.zeros(J)
        _check(lib().cfr_get_values(self._h, game, player, _ptr(x), _ptr(ev)), "cfr_get_values")
        return {"x": x, "ev": ev}

    def set_state(self, player: int, r, b, xbar, t: int, game: int = 0):
        S = self._game_sizes(game)["S1" if player == 1 else "S2"]
        r = np.ascontiguousarray(r, np.float64)
        b = np.ascontiguousarray(b, np.float64)
        xbar = np.ascontiguousarray(xbar, np.float64)
        if r.shape[0] != S or b.shape[0] != S or xbar.shape[0] != S + 1:
            raise ValueError("state vectors must have lengths S, S, S + 1")
        _check(lib().cfr_set_state(self._h, game, player, _ptr(r), _ptr(b), _ptr(xbar), int(t)),
               "cfr_set_state")
