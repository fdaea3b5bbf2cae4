"""ctypes binding of ``libprot.so`` (the C ABI declared in ``include/prot.h``).

Argument marshalling only: every step of the solver runs in the CUDA library.
There is no CPU fallback; if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_PKG, "libprot.so")

PR_OK = 0
PR_ERR_INVALID = -1
PR_ERR_CUDA = -2
PR_ERR_TIMEOUT = -3
PR_ERR_NO_CONVERGENCE = -4
PR_ERR_WORKSPACE = -5
PR_ERR_CAPACITY = -6
PR_ERR_INTERNAL = -7
PR_F32 = 0
PR_F64 = 1


class PrStats(ctypes.Structure):
    _fields_ = [
        ("phases", ctypes.c_int64),
        ("rounds", ctypes.c_int64),
        ("bytes_scanned", ctypes.c_int64),
        ("rows_scanned", ctypes.c_int64),
        ("free_at_stop", ctypes.c_int32),
        ("threshold", ctypes.c_int32),
        ("loop_ctas", ctypes.c_int32),
        ("loop_cluster", ctypes.c_int32),
        ("cells_examined", ctypes.c_int64),
        ("barriers", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PrBatchedTune(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


PR_RULE_LOWEST = 0
PR_RULE_OFFSET = 1
PR_RULE_ISRAELI_ITAI = 2
PR_RULE_SEQUENTIAL = 3

PR_SQEUCLIDEAN = 0
PR_EUCLIDEAN = 1


class PrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_sz = ctypes.c_size_t

# name -> (restype, argtypes); every symbol include/prot.h declares.
SIGNATURES = {
    "pr_assign_workspace": (_sz, [_i32, _i32]),
    "pr_assign_within": (ctypes.c_int, [_vp, ctypes.c_int, _i64, _i32, _i32, _dbl, _vp, _vp, _vp, _vp, _vp,
                                        ctypes.POINTER(PrStats), _vp, _sz, _vp]),
    "pr_probe_workspace": (_sz, []),
    "pr_probe_latency": (ctypes.c_int, [_vp, _sz, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), _vp]),
    "pr_assign": (ctypes.c_int, [_vp, ctypes.c_int, _i64, _i32, _i32, _dbl, _vp, _vp, _vp, _vp, _vp,
                                 ctypes.POINTER(PrStats), _vp, _sz, _vp]),
    "pr_assign_batched_workspace": (_sz, [_i32, _vp]),
    "pr_assign_batched": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _vp, _dbl, _vp, _vp, _vp, _vp, _vp,
                                         _vp, ctypes.POINTER(PrBatchedTune), ctypes.POINTER(PrStats),
                                         _vp, _sz, _vp]),
    "pr_assign_batched_points": (ctypes.c_int, [_vp, _vp, _i32, ctypes.c_int, _i32, _vp, _dbl, _vp, _vp,
                                                _vp, _vp, _vp, _vp, ctypes.POINTER(PrBatchedTune),
                                                ctypes.POINTER(PrStats), _vp, _sz, _vp]),
    "pr_ot_workspace": (_sz, [_i32, _i32]),
    "pr_ot": (ctypes.c_int, [_vp, ctypes.c_int, _i64, _i32, _i32, _vp, _vp, _dbl, _i64, _vp, _vp, _vp, _vp,
                             _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(PrStats), _vp, _sz, _vp]),
    "pr_assign_backward": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
    "pr_assign_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _i64, _i32, _i32, _dbl, _vp, _vp, _vp, _vp,
                                         _vp, ctypes.POINTER(PrStats), _vp]),
    "pr_assign_batched_autotune": (ctypes.c_int, [_vp, _vp, _i32, ctypes.c_int, _vp, ctypes.c_int, _i32, _vp,
                                                  _dbl, _vp, _vp, _vp, _vp, _vp, _vp,
                                                  ctypes.POINTER(PrBatchedTune), ctypes.POINTER(ctypes.c_float),
                                                  _vp, _sz, _vp]),
    "pr_dual_bound": (ctypes.c_int, [_vp, _vp, _i32, _i32, _dbl, _vp, _vp, _vp]),
    "pr_assign_rule": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.c_int, _i64, _i32, _i32, _dbl, _vp, _vp, _vp,
                                      _vp, _vp, ctypes.POINTER(PrStats), _vp, _sz, _vp]),
    "pr_assign_staged": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _i64, _i32, _i32, _dbl, _vp, _vp, _vp, _vp,
                                        _vp, ctypes.POINTER(PrStats), _vp, _sz, _vp]),
    "pr_assign_points": (ctypes.c_int, [_vp, _vp, _i32, ctypes.c_int, _i32, _i32, _dbl, _vp, _vp, _vp, _vp,
                                        _vp, ctypes.POINTER(PrStats), _vp, _sz, _vp]),
    "pr_ws_status": (ctypes.c_int, [_vp, _vp]),
    "pr_set_kernel_events": (None, [_vp, _vp]),
    "pr_last_error": (ctypes.c_char_p, []),
    "pr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def load(path: str = SO_PATH):
    """Load the CUDA library; raises if it was not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(
                    f"{path} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                if hasattr(L, name):
                    fn = getattr(L, name)
                    fn.restype = res
                    fn.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str):
    if status != PR_OK:
        msg = load().pr_last_error().decode(errors="replace")
        raise PrError(status, f"{what}: {msg}")
