"""ctypes binding of libvomt (the C ABI declared in include/vomt.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
If the library is missing or cannot be built this module raises; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_double, c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
P_int, P_double, P_float = ctypes.POINTER(c_int), ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_float)

OK, NOT_CONVERGED = 0, 1
TAU_GRID = 10         # VOMT_TAU_GRID
STATUS_NAMES = {
    0: "OK", 1: "NOT_CONVERGED", -1: "BAD_ARG", -2: "MASS_MISMATCH", -3: "NEGATIVE_DENSITY",
    -4: "GRAPH", -5: "L_KERNEL", -6: "STEP_CONDITION", -7: "NONFINITE", -8: "BARRIER_TIMEOUT",
    -9: "CUDA", -10: "TOO_LARGE",
}
ENGINES = {"auto": 0, "stream": 1, "resident": 2, "batched": 3}
ENGINE_NAMES = {v: k for k, v in ENGINES.items()}


class Graph(ctypes.Structure):
    _fields_ = [("k", c_int), ("n_edges", c_int), ("tail", P_int), ("head", P_int), ("cost", P_double)]


class Instance(ctypes.Structure):
    _fields_ = [("n", c_int), ("graph", Graph), ("alpha", c_double), ("tau", c_double), ("offset", ctypes.c_size_t)]


class Params(ctypes.Structure):
    _fields_ = [("tau", c_double), ("mu", c_double), ("nu", c_double), ("u_norm", c_int), ("w_norm", c_int),
                ("max_iters", c_int), ("check_every", c_int), ("tol_gap", c_double), ("tol_res", c_double),
                ("warm_start", c_int), ("engine", c_int), ("halo", c_int), ("eps", c_double), ("pitch", c_int)]


class Result(ctypes.Structure):
    _fields_ = [("primal", c_double), ("dual", c_double), ("rel_gap", c_double), ("rel_res", c_double),
                ("fp_resid", c_double), ("dual_infeas", c_double), ("mu", c_double), ("nu", c_double),
                ("tau", c_double), ("iters", c_int), ("status", c_int), ("engine", c_int), ("checks", c_int),
                ("launches", c_int), ("blocks", c_int), ("halo", c_int), ("variant", c_int)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["engine"] = ENGINE_NAMES.get(d["engine"], d["engine"])
        return d


class VomtError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, message))
        self.status = status


# every symbol include/vomt.h declares, with its ctypes signature
SIGNATURES = {
    "vomt_create": (c_int, [ctypes.POINTER(c_void_p), c_int]),
    "vomt_destroy": (None, [c_void_p]),
    "vomt_status_str": (ctypes.c_char_p, [c_int]),
    "vomt_last_error": (ctypes.c_char_p, [c_void_p]),
    "vomt_default_params": (None, [ctypes.POINTER(Params)]),
    "vomt_step_sizes": (c_int, [c_int, ctypes.POINTER(Graph), c_double, P_double, P_double, P_double, P_double]),
    "vomt_solve": (c_int, [c_void_p, c_int, c_void_p, c_void_p, ctypes.POINTER(Graph), c_double,
                           ctypes.POINTER(Params), c_void_p, c_void_p, c_void_p, ctypes.POINTER(Result), c_void_p]),
    "vomt_solve_host": (c_int, [c_void_p, c_int, c_void_p, c_void_p, ctypes.POINTER(Graph), c_double,
                                ctypes.POINTER(Params), c_void_p, c_void_p, c_void_p, ctypes.POINTER(Result),
                                c_void_p]),
    "vomt_solve3d": (c_int, [c_void_p, c_int, c_void_p, c_void_p, ctypes.POINTER(Graph), c_double,
                             ctypes.POINTER(Params), c_void_p, c_void_p, c_void_p, ctypes.POINTER(Result), c_void_p]),
    "momt_solve_complex": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int, c_void_p, c_double,
                                   ctypes.POINTER(Params), c_void_p, c_void_p, c_void_p, ctypes.POINTER(Result),
                                   c_void_p]),
    "momt_solve3d": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int, c_void_p, c_double,
                             ctypes.POINTER(Params), c_void_p, c_void_p, c_void_p, ctypes.POINTER(Result), c_void_p]),
    "vomt_history": (c_int, [c_void_p, P_double, c_int]),
    "vomt_set_wait_policy": (c_int, [c_void_p, c_double, c_int]),
    "vomt_backward": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_void_p, c_void_p, c_void_p]),
    "vomt_unrolled_grad": (c_int, [c_void_p, c_int, c_void_p, c_void_p, ctypes.POINTER(Graph), c_double,
                                   ctypes.POINTER(Params), c_int, c_int, c_double, c_void_p, c_void_p, P_double,
                                   P_double, c_void_p]),
    "vomt_batch_layout": (c_int, [c_int, ctypes.POINTER(Instance), ctypes.POINTER(ctypes.c_size_t)]),
    "vomt_solve_batched": (c_int, [c_void_p, c_int, ctypes.POINTER(Instance), c_void_p, ctypes.POINTER(Params),
                                   ctypes.POINTER(Result), c_void_p]),
    "vomt_batch_tune": (c_int, [c_void_p, c_int, ctypes.POINTER(Instance), c_void_p, ctypes.POINTER(Params), c_int,
                                P_int, P_double]),
    "vomt_batch_set_threads": (c_int, [c_void_p, c_int]),
    "momt_step_sizes": (c_int, [c_int, c_int, c_int, c_void_p, c_double, P_double, P_double, P_double, P_double,
                                P_double]),
    "momt_solve": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int, c_void_p, c_double,
                           ctypes.POINTER(Params), c_void_p, c_void_p, c_void_p, ctypes.POINTER(Result), c_void_p]),
    "vomt_tune_tau": (c_int, [c_void_p, c_int, c_void_p, c_void_p, ctypes.POINTER(Graph), c_double,
                              ctypes.POINTER(Params), c_int, c_void_p, c_void_p, c_void_p, P_double, P_double,
                              P_double, c_void_p]),
    "momt_tune_tau": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int, c_void_p, c_double,
                              ctypes.POINTER(Params), c_int, c_void_p, c_void_p, c_void_p, P_double, P_double,
                              P_double, c_void_p]),
    "vomt_batch_tune_tau": (c_int, [c_void_p, c_int, ctypes.POINTER(Instance), c_void_p, ctypes.POINTER(Params),
                                    c_int, P_double, P_double]),
    "vomt_solve_noalloc": (c_int, [c_int, c_void_p, c_void_p, ctypes.POINTER(Graph), c_double,
                                   ctypes.POINTER(Params), c_void_p, c_void_p, c_void_p, ctypes.POINTER(Result),
                                   c_void_p, ctypes.POINTER(ctypes.c_char_p)]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libvomt.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libvomt.so is missing; build it with `python -m paper_1712_10279_gb300.build`")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


_contexts = {}


def context(device: int = 0):
    lib = load()
    ctx = _contexts.get(device)
    if ctx is None:
        h = c_void_p()
        rc = lib.vomt_create(ctypes.byref(h), device)
        if rc != 0:
            raise VomtError(rc, "vomt_create failed on device %d" % device)
        ctx = h
        _contexts[device] = ctx
    return ctx


def check(rc, ctx=None):
    if rc < 0:
        lib = load()
        msg = lib.vomt_last_error(ctx).decode() if ctx else lib.vomt_status_str(rc).decode()
        raise VomtError(rc, msg)
    return rc


class GraphArg:
    """Keeps the edge arrays alive while the C call runs."""

    def __init__(self, k, edges, cost=None):
        import numpy as np
        e = np.asarray(list(edges), dtype=np.int32).reshape(-1, 2)
        self.tail = np.ascontiguousarray(e[:, 0])
        self.head = np.ascontiguousarray(e[:, 1])
        self.cost = None if cost is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(cost, np.float64), (e.shape[0],)))
        self.g = Graph(int(k), int(e.shape[0]),
                       self.tail.ctypes.data_as(P_int) if e.shape[0] else None,
                       self.head.ctypes.data_as(P_int) if e.shape[0] else None,
                       self.cost.ctypes.data_as(P_double) if self.cost is not None else None)

    @property
    def ref(self):
        return ctypes.byref(self.g)
