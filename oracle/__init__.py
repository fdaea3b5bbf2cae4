"""CPU oracle for the push-relabel additive approximation (arXiv 2203.03732).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's ``cpu_baseline`` / ``--impl reference`` legs may use this package;
the product library never does.  The C sources here share nothing with the
CUDA path; this module only compiles them with gcc and marshals numpy arrays
through ctypes.

Functions follow the paper's steps (Sec. 2.2 phase loop, Eq. 1 rounding,
Sec. 2.1 completion); see ``prot_oracle.c`` for the citations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["prot_oracle.c", "ot_oracle.c", "points_oracle.c"]
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID = -1
ERR_NO_CONVERGENCE = -4

MODE_RESUME = 0
MODE_LITERAL = 1
MODE_CHECK = 2
MODE_REVERSE = 4
MODE_SEQUENTIAL = 8
MODE_EVICT_RESUME = 16
MODE_OFFSET = 32
MODE_PARALLEL = 64
MODE_ISRAELI_ITAI = 128


class Stats(ctypes.Structure):
    _fields_ = [
        ("phases", ctypes.c_int64),
        ("rounds", ctypes.c_int64),
        ("scanned", ctypes.c_int64),
        ("sum_ni", ctypes.c_int64),
        ("violations", ctypes.c_int64),
        ("free_at_stop", ctypes.c_int32),
        ("threshold", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle into ``liboracle.so`` (plain gcc, no CUDA)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        deps = srcs + [os.path.join(_HERE, h) for h in os.listdir(_HERE) if h.endswith(".h")]
        if all(os.path.getmtime(s) <= so_t for s in deps):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-fopenmp", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            _declare(L)
            _lib = L
    return _lib


_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


def _declare(L):
    c_i32, c_i64, c_dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.or_quantise_f64.argtypes = [_f64p, c_i64, c_i32, c_i32, c_dbl, _i32p]
    L.or_quantise_f64.restype = ctypes.c_int
    L.or_quantise_f32.argtypes = [_f32p, c_i64, c_i32, c_i32, c_dbl, _i32p]
    L.or_quantise_f32.restype = ctypes.c_int
    L.or_threshold.argtypes = [c_dbl, c_i32]
    L.or_threshold.restype = c_i32
    L.or_phase_cap.argtypes = [c_dbl, c_i32]
    L.or_phase_cap.restype = c_i64
    L.or_check_state.argtypes = [_i32p, c_i32, c_i32, _i32p, _i32p, _i32p, _i32p]
    L.or_check_state.restype = c_i64
    L.or_assign_int.argtypes = [_i32p, c_i32, c_i32, c_i32, c_i32, c_i64, _i32p, _i32p, _i32p,
                                _i32p, ctypes.POINTER(Stats), ctypes.c_void_p, c_i64]
    L.or_assign_int.restype = ctypes.c_int
    L.or_complete.argtypes = [c_i32, c_i32, _i32p, _i32p]
    L.or_complete.restype = None
    L.or_cost_f64.argtypes = [_f64p, c_i64, c_i32, _i32p]
    L.or_cost_f64.restype = c_dbl
    L.or_cost_f32.argtypes = [_f32p, c_i64, c_i32, _i32p]
    L.or_cost_f32.restype = c_dbl
    L.or_hungarian.argtypes = [_f64p, c_i64, c_i32, c_i32, _i32p]
    L.or_hungarian.restype = c_dbl
    L.or_ii_key.argtypes = [ctypes.c_uint32] * 5
    L.or_ii_key.restype = ctypes.c_uint64
    if hasattr(L, "or_ot_cluster_int"):
        from . import ot as _ot
        _ot._declare(L)
    if hasattr(L, "or_assign_points"):
        from . import points as _pts
        _pts._declare(L)


# --------------------------------------------------------------------------
# Assignment (Sec. 2.2)
# --------------------------------------------------------------------------

def quantise(C: np.ndarray, eps: float) -> np.ndarray:
    """Eq. (1) in eps units: cb = floor of the exact quotient C / eps, int32."""
    C = np.ascontiguousarray(C)
    nB, nA = C.shape
    cb = np.empty((nB, nA), dtype=np.int32)
    if C.dtype == np.float64:
        rc = lib().or_quantise_f64(C, nA, nB, nA, float(eps), cb)
    elif C.dtype == np.float32:
        rc = lib().or_quantise_f32(C, nA, nB, nA, float(eps), cb)
    else:
        raise TypeError(C.dtype)
    if rc != 0:
        raise ValueError("costs must be finite and in [0, 1]")
    return cb


def threshold(eps: float, nB: int) -> int:
    return int(lib().or_threshold(float(eps), int(nB)))


def phase_cap(eps: float, nB: int) -> int:
    return int(lib().or_phase_cap(float(eps), int(nB)))


def assign_int(cb: np.ndarray, T: int, mode: int = MODE_RESUME, phase_cap_: int | None = None,
               eps_for_cap: float | None = None, ni_log: bool = False):
    """Main routine of Sec. 2.2 on integer costs (before completion).

    Returns dict(match_b, match_a, y_b, y_a, stats, rc[, ni]).
    """
    cb = np.ascontiguousarray(cb, dtype=np.int32)
    nB, nA = cb.shape
    if phase_cap_ is None:
        phase_cap_ = phase_cap(eps_for_cap, nB) if eps_for_cap is not None else 1 << 40
    mb = np.empty(nB, np.int32)
    ma = np.empty(nA, np.int32)
    yb = np.empty(nB, np.int32)
    ya = np.empty(nA, np.int32)
    st = Stats()
    log = np.zeros(1 << 16, np.int32) if ni_log else None
    rc = lib().or_assign_int(cb, nB, nA, int(T), int(mode), int(phase_cap_), mb, ma, yb, ya,
                             ctypes.byref(st),
                             log.ctypes.data_as(ctypes.c_void_p) if ni_log else None,
                             int(log.size) if ni_log else 0)
    out = dict(match_b=mb, match_a=ma, y_b=yb, y_a=ya, stats=st.as_dict(), rc=rc)
    if ni_log:
        out["ni"] = log[: min(st.phases, log.size)].copy()
    return out


def complete(match_b: np.ndarray, match_a: np.ndarray):
    """Sec. 2.1 completion: k-th free b with the k-th free a (in place)."""
    lib().or_complete(match_b.size, match_a.size, match_b, match_a)


def cost(C: np.ndarray, match_b: np.ndarray) -> float:
    C = np.ascontiguousarray(C)
    nB, nA = C.shape
    if C.dtype == np.float64:
        return float(lib().or_cost_f64(C, nA, nB, np.ascontiguousarray(match_b, np.int32)))
    return float(lib().or_cost_f32(C, nA, nB, np.ascontiguousarray(match_b, np.int32)))


def assign(C: np.ndarray, eps: float, mode: int = MODE_RESUME):
    """Whole oracle solve: Eq. (1), Sec. 2.2 main routine, completion, c(M).

    Returns dict(row_to_col, col_to_row, y_row, y_col, cost, stats) with the
    duals in units of eps (integers)."""
    C = np.ascontiguousarray(C)
    if C.dtype not in (np.float64, np.float32):
        raise TypeError(C.dtype)
    nB, nA = C.shape
    if not (0.0 < eps < 1.0) or np.floor(1.0 / eps) > 32766:
        raise ValueError("eps out of range")
    cb = quantise(C, eps)
    T = threshold(eps, nB)
    r = assign_int(cb, T, mode=mode, phase_cap_=phase_cap(eps, nB))
    if r["rc"] != OK:
        raise RuntimeError(f"oracle failed rc={r['rc']}")
    complete(r["match_b"], r["match_a"])
    c = cost(C, r["match_b"])
    return dict(row_to_col=r["match_b"], col_to_row=r["match_a"], y_row=r["y_b"],
                y_col=r["y_a"], cost=c, stats=r["stats"], cbar=cb, threshold=T)


def ii_key(step: int, phase: int, it: int, u: int, v: int) -> int:
    """Key of candidate v for vertex u in the randomized rule's step `step`
    (see prot_oracle.c): 40 random bits above the 24-bit candidate index."""
    return int(lib().or_ii_key(step, phase, it, u, v))


def check_state(cb, match_b, match_a, y_b, y_a) -> int:
    cb = np.ascontiguousarray(cb, np.int32)
    nB, nA = cb.shape
    return int(lib().or_check_state(cb, nB, nA, np.ascontiguousarray(match_b, np.int32),
                                    np.ascontiguousarray(match_a, np.int32),
                                    np.ascontiguousarray(y_b, np.int32),
                                    np.ascontiguousarray(y_a, np.int32)))


def hungarian(C: np.ndarray):
    """Exact minimum-cost assignment (rows <= cols).  Returns (cost, row_to_col)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    nB, nA = C.shape
    r2c = np.empty(nB, np.int32)
    v = lib().or_hungarian(C, nA, nB, nA, r2c)
    return float(v), r2c
