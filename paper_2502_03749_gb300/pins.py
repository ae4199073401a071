"""Python binding of the PINS C ABI (include/pins.h).

Argument marshalling only: every step of the solver runs in libpins.so.  The
functions keep the C names (pins_create, pins_solve, ...); `Pins` wraps a handle
for convenience.  Arrays may be NumPy arrays (host) or torch CUDA tensors
(device; float64, contiguous).  If the library is missing or the CUDA device
is unavailable, calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpins.so")

PINS_OK = 0
PINS_ERR_INVALID_ARG = 1
PINS_ERR_OOM = 2
PINS_ERR_NOT_CONVERGED = 3
PINS_ERR_LINESEARCH = 4
PINS_ERR_QUEUE_FULL = 5
PINS_ERR_PENDING = 6
PINS_ERR_CUDA = 7
PINS_ERR_UNKNOWN_TICKET = 8
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "NOT_CONVERGED", 4: "LINESEARCH",
                5: "QUEUE_FULL", 6: "PENDING", 7: "CUDA", 8: "UNKNOWN_TICKET"}

PINS_COST_DENSE_F64 = 0
PINS_COST_DENSE_F32 = 1
PINS_COST_POINTS_SQEUCLID = 2
PINS_COST_GRID_SQEUCLID = 3
PINS_PREC_FP64 = 0
PINS_PREC_MIXED = 1

EXPORTED = ["pins_config_default", "pins_create", "pins_destroy", "pins_last_error",
            "pins_solve", "pins_solve_batch", "pins_submit", "pins_poll", "pins_wait",
            "pins_step_sinkhorn", "pins_step_marginals", "pins_step_sparsify", "pins_step_cg",
            "pins_step_objective_increase", "pins_step_certificate", "pins_profile_classes",
            "pins_profile_name", "pins_profile_read", "pins_marginals_noalloc",
            "pins_serving_held_bytes", "pins_test_inject_faults"]


class pins_config(ct.Structure):
    _fields_ = [("eta", ct.c_double), ("tol_marg", ct.c_double), ("tol_gap", ct.c_double),
                ("cg_rtol", ct.c_double), ("armijo_beta", ct.c_double),
                ("armijo_c1", ct.c_double), ("sparsify_gamma", ct.c_double),
                ("T1", ct.c_int), ("T2", ct.c_int), ("K", ct.c_int), ("max_cg", ct.c_int),
                ("max_backtrack", ct.c_int), ("sinkhorn_check_every", ct.c_int),
                ("gap_every", ct.c_int), ("prec", ct.c_int), ("device", ct.c_int),
                ("cuda_stream", ct.c_void_p), ("max_inflight", ct.c_int),
                ("queue_capacity", ct.c_int), ("device_mem_budget", ct.c_size_t),
                ("profile", ct.c_int), ("sparsify_one_pass", ct.c_int)]


class pins_problem(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("m", ct.c_int), ("n", ct.c_int), ("d", ct.c_int),
                ("C", ct.c_void_p), ("x", ct.c_void_p), ("y", ct.c_void_p),
                ("cost_scale", ct.c_double), ("grid_s1", ct.c_int), ("grid_s2", ct.c_int),
                ("a", ct.c_void_p), ("b", ct.c_void_p), ("on_device", ct.c_int)]


class pins_result(ct.Structure):
    _fields_ = [("status", ct.c_int), ("cost", ct.c_double), ("cost_ub", ct.c_double),
                ("dual_lb", ct.c_double), ("rel_gap", ct.c_double),
                ("marg_resid_l1", ct.c_double), ("s", ct.c_double),
                ("outer_iters", ct.c_int), ("sinkhorn_iters", ct.c_int),
                ("newton_iters", ct.c_int), ("cg_iters", ct.c_int), ("ls_trials", ct.c_int),
                ("ls_failures", ct.c_int), ("gpu_launches", ct.c_int),
                ("seconds", ct.c_double), ("F_out", ct.c_void_p), ("G_out", ct.c_void_p)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k not in ("F_out", "G_out")}


_lib = None


def load(path: str = LIB_PATH) -> ct.CDLL:
    """Loads libpins.so; raises if it is absent (build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ct.CDLL(path)
    P = ct.c_void_p
    D = ct.c_double
    I = ct.c_int
    lib.pins_config_default.argtypes = [ct.POINTER(pins_config)]
    lib.pins_config_default.restype = None
    lib.pins_create.argtypes = [ct.POINTER(pins_config), ct.POINTER(P)]
    lib.pins_destroy.argtypes = [P]
    lib.pins_destroy.restype = None
    lib.pins_last_error.argtypes = [P]
    lib.pins_last_error.restype = ct.c_char_p
    lib.pins_solve.argtypes = [P, ct.POINTER(pins_problem), ct.POINTER(pins_result)]
    lib.pins_solve_batch.argtypes = [P, ct.POINTER(pins_problem), I, ct.POINTER(pins_result)]
    lib.pins_submit.argtypes = [P, ct.POINTER(pins_problem), ct.POINTER(ct.c_uint64)]
    lib.pins_poll.argtypes = [P, ct.c_uint64, ct.POINTER(pins_result)]
    lib.pins_wait.argtypes = [P, ct.c_uint64, ct.POINTER(pins_result)]
    lib.pins_step_sinkhorn.argtypes = [P, ct.POINTER(pins_problem), D, I, P, P, P]
    lib.pins_step_marginals.argtypes = [P, ct.POINTER(pins_problem), D, P, P, P, P, P]
    lib.pins_step_sparsify.argtypes = [P, ct.POINTER(pins_problem), D, P, P, I, P, P, P]
    lib.pins_step_cg.argtypes = [P, I, I, D, P, P, P, P, P, I, P, P, D, I, P]
    lib.pins_step_objective_increase.argtypes = [P, ct.POINTER(pins_problem), D, P, P, P, P,
                                                 D, P]
    lib.pins_step_certificate.argtypes = [P, ct.POINTER(pins_problem), D, P, P, P]
    lib.pins_profile_classes.argtypes = []
    lib.pins_profile_name.argtypes = [I]
    lib.pins_profile_read.argtypes = [P, P, P, I, I]
    lib.pins_marginals_noalloc.argtypes = [ct.POINTER(pins_problem), D, I, D, P, P, P, P, P, P]
    lib.pins_serving_held_bytes.argtypes = [P, ct.POINTER(ct.c_size_t), ct.POINTER(ct.c_size_t)]
    lib.pins_test_inject_faults.argtypes = [P, I, I, I]
    for name in EXPORTED:
        if name not in ("pins_config_default", "pins_destroy", "pins_last_error"):
            getattr(lib, name).restype = ct.c_int
    lib.pins_profile_name.restype = ct.c_char_p
    _lib = lib
    return lib


# --------------------------------------------------------------------------- #
# Same-name wrappers of the C functions
# --------------------------------------------------------------------------- #
def pins_config_default() -> pins_config:
    c = pins_config()
    load().pins_config_default(ct.byref(c))
    return c


def pins_create(cfg: pins_config) -> ct.c_void_p:
    h = ct.c_void_p()
    st = load().pins_create(ct.byref(cfg), ct.byref(h))
    if st != PINS_OK:
        raise RuntimeError(f"pins_create failed: {STATUS_NAMES.get(st, st)}")
    return h


def pins_destroy(h) -> None:
    load().pins_destroy(h)


def pins_last_error(h) -> str:
    return load().pins_last_error(h).decode()


def pins_solve(h, prob: pins_problem, res: pins_result) -> int:
    return load().pins_solve(h, ct.byref(prob), ct.byref(res))


def pins_solve_batch(h, probs, res) -> int:
    return load().pins_solve_batch(h, probs, len(probs), res)


def pins_submit(h, prob: pins_problem) -> tuple:
    t = ct.c_uint64()
    st = load().pins_submit(h, ct.byref(prob), ct.byref(t))
    return st, t.value


def pins_poll(h, ticket: int, res: pins_result) -> int:
    return load().pins_poll(h, ct.c_uint64(ticket), ct.byref(res))


def pins_wait(h, ticket: int, res: pins_result) -> int:
    return load().pins_wait(h, ct.c_uint64(ticket), ct.byref(res))


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def pins_step_sinkhorn(h, prob, s, iters, F, G, row_res=None) -> int:
    return load().pins_step_sinkhorn(h, ct.byref(prob), s, iters, _ptr(F), _ptr(G), _ptr(row_res))


def pins_step_marginals(h, prob, s, F, G, r, c, out3) -> int:
    return load().pins_step_marginals(h, ct.byref(prob), s, _ptr(F), _ptr(G), _ptr(r), _ptr(c),
                                      _ptr(out3))


def pins_step_sparsify(h, prob, s, F, G, keep, indptr, indices, data) -> int:
    return load().pins_step_sparsify(h, ct.byref(prob), s, _ptr(F), _ptr(G), keep,
                                     _ptr(indptr), _ptr(indices), _ptr(data))


def pins_step_cg(h, m, n, eta, r, c, indptr, indices, data, nnz, rhs, d, rtol, max_iter,
                 info) -> int:
    return load().pins_step_cg(h, m, n, eta, _ptr(r), _ptr(c), _ptr(indptr), _ptr(indices),
                               _ptr(data), nnz, _ptr(rhs), _ptr(d), rtol, max_iter, _ptr(info))


def pins_step_objective_increase(h, prob, s, F, G, df, dg, alpha, out) -> int:
    return load().pins_step_objective_increase(h, ct.byref(prob), s, _ptr(F), _ptr(G), _ptr(df),
                                               _ptr(dg), alpha, _ptr(out))


def pins_step_certificate(h, prob, s, F, G, out6) -> int:
    return load().pins_step_certificate(h, ct.byref(prob), s, _ptr(F), _ptr(G), _ptr(out6))


def pins_marginals_noalloc(prob, eta, prec, s, F, G, r, c, out3, stream=None) -> int:
    """Allocation-free marginal pass (see include/pins.h); queued on `stream`."""
    return load().pins_marginals_noalloc(ct.byref(prob), eta, prec, s, _ptr(F), _ptr(G),
                                         _ptr(r), _ptr(c), _ptr(out3), stream)


def pins_serving_held_bytes(h):
    """(bytes held by the serving pool's arenas, admission budget)."""
    held, budget = ct.c_size_t(0), ct.c_size_t(0)
    st = load().pins_serving_held_bytes(h, ct.byref(held), ct.byref(budget))
    if st != PINS_OK:
        raise RuntimeError(f"pins_serving_held_bytes: {STATUS_NAMES.get(st, st)}")
    return int(held.value), int(budget.value)


def pins_test_inject_faults(h, alloc_failures: int, kernel_errors: int,
                            selection_failures: int = 0) -> int:
    return load().pins_test_inject_faults(h, alloc_failures, kernel_errors, selection_failures)


def pins_profile_classes() -> int:
    return load().pins_profile_classes()


def pins_profile_name(k: int) -> str:
    return load().pins_profile_name(k).decode()


def pins_profile_read(h, reset: bool = False) -> dict:
    """{class name: (device ms, launches)} of the handle's blocking solver."""
    n = pins_profile_classes()
    ms = (ct.c_double * n)()
    cnt = (ct.c_longlong * n)()
    load().pins_profile_read(h, ms, cnt, n, 1 if reset else 0)
    return {pins_profile_name(k): (ms[k], cnt[k]) for k in range(n)}


# --------------------------------------------------------------------------- #
# Problem construction and a handle wrapper
# --------------------------------------------------------------------------- #
class ProblemRef:
    """A pins_problem plus references that keep its arrays alive."""

    def __init__(self, prob: pins_problem, keep: Sequence):
        self.prob = prob
        self.keep = list(keep)


def make_problem(kind: str, a, b, C=None, x=None, y=None, cost_scale: float = 1.0,
                 grid=(0, 0), on_device: bool = False) -> ProblemRef:
    """kind: 'dense' (C float64 or float32), 'points' (x: m x d, y: n x d float64),
    'grid' (grid = (s1, s2)).  Host arrays are NumPy; device arrays torch CUDA tensors."""
    keep = []

    def arr(v, dtype):
        if v is None:
            return None
        if hasattr(v, "data_ptr"):
            assert v.is_contiguous()
            keep.append(v)
            return v.data_ptr()
        v = np.ascontiguousarray(v, dtype=dtype)
        keep.append(v)
        return v.ctypes.data

    p = pins_problem()
    p.m = int(a.shape[0])
    p.n = int(b.shape[0])
    p.a = arr(a, np.float64)
    p.b = arr(b, np.float64)
    p.on_device = 1 if on_device else 0
    p.cost_scale = float(cost_scale)
    if kind == "dense":
        is32 = (str(C.dtype) in ("float32", "torch.float32"))
        p.kind = PINS_COST_DENSE_F32 if is32 else PINS_COST_DENSE_F64
        p.C = arr(C, np.float32 if is32 else np.float64)
    elif kind == "points":
        p.kind = PINS_COST_POINTS_SQEUCLID
        p.d = int(x.shape[1])
        p.x = arr(x, np.float64)
        p.y = arr(y, np.float64)
    elif kind == "grid":
        p.kind = PINS_COST_GRID_SQEUCLID
        p.grid_s1, p.grid_s2 = int(grid[0]), int(grid[1])
    else:
        raise ValueError(kind)
    return ProblemRef(p, keep)


def problem_from_workload(w, as_kind: Optional[str] = None) -> ProblemRef:
    """Builds a host problem from paper_2502_03749_gb300.workloads.Problem."""
    kind = as_kind or w.kind
    if kind == "dense":
        return make_problem("dense", w.a, w.b, C=w.dense_cost())
    if kind == "points":
        return make_problem("points", w.a, w.b, x=w.x, y=w.y, cost_scale=w.cost_scale)
    return make_problem("grid", w.a, w.b, cost_scale=w.cost_scale, grid=w.grid)


class Pins:
    """Handle wrapper: Pins(eta=..., prec='fp64'|'mixed', ...).solve(problem_ref)."""

    def __init__(self, **cfg):
        c = pins_config_default()
        prec = cfg.pop("prec", "fp64")
        c.prec = PINS_PREC_MIXED if prec in ("mixed", PINS_PREC_MIXED) else PINS_PREC_FP64
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise KeyError(k)
            setattr(c, k, v)
        self.cfg = c
        self.h = pins_create(c)

    def close(self):
        if self.h is not None:
            pins_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return pins_last_error(self.h)

    def solve(self, pref: ProblemRef, want_potentials: bool = True) -> dict:
        res = pins_result()
        F = np.zeros(pref.prob.m) if want_potentials else None
        G = np.zeros(pref.prob.n) if want_potentials else None
        if want_potentials:
            res.F_out = F.ctypes.data
            res.G_out = G.ctypes.data
        st = pins_solve(self.h, pref.prob, res)
        if st not in (PINS_OK, PINS_ERR_NOT_CONVERGED):
            raise RuntimeError(f"pins_solve: {STATUS_NAMES.get(st, st)}: {self.error()}")
        out = res.as_dict()
        out["F"], out["G"] = F, G
        return out

    def solve_batch(self, prefs: Sequence[ProblemRef]) -> list:
        n = len(prefs)
        probs = (pins_problem * n)(*[p.prob for p in prefs])
        res = (pins_result * n)()
        Fs = [np.zeros(p.prob.m) for p in prefs]
        Gs = [np.zeros(p.prob.n) for p in prefs]
        for i in range(n):
            res[i].F_out = Fs[i].ctypes.data
            res[i].G_out = Gs[i].ctypes.data
        load().pins_solve_batch(self.h, probs, n, res)
        out = []
        for i in range(n):
            d = res[i].as_dict()
            d["F"], d["G"] = Fs[i], Gs[i]
            out.append(d)
        return out

    def submit(self, pref: ProblemRef) -> int:
        st, t = pins_submit(self.h, pref.prob)
        if st != PINS_OK:
            raise RuntimeError(f"pins_submit: {STATUS_NAMES.get(st, st)}: {self.error()}")
        return t

    def poll(self, ticket: int, potentials: Optional[tuple] = None):
        res = pins_result()
        if potentials is not None:
            res.F_out = potentials[0].ctypes.data
            res.G_out = potentials[1].ctypes.data
        st = pins_poll(self.h, ticket, res)
        if st == PINS_ERR_PENDING:
            return None
        d = res.as_dict()
        d["status"] = st
        return d

    def wait(self, ticket: int, potentials: Optional[tuple] = None) -> dict:
        res = pins_result()
        if potentials is not None:
            res.F_out = potentials[0].ctypes.data
            res.G_out = potentials[1].ctypes.data
        st = pins_wait(self.h, ticket, res)
        d = res.as_dict()
        d["status"] = st
        return d
