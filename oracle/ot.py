"""Oracle wrappers for the optimal-transport form (Sec. 4), test infrastructure
only: mass quantisation, the cluster phase loop, the plan and its fix-up."""
from __future__ import annotations

import ctypes

import numpy as np

from . import Stats, lib, OK, quantise, phase_cap as _phase_cap

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _declare(L):
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.or_ot_cluster_int.argtypes = [_i32p, i32, i32, _i32p, _i32p, i64, i32, i64, _i32p, _i32p,
                                    _i32p, _i32p, _i32p, _i32p, _i32p, ctypes.POINTER(Stats)]
    L.or_ot_cluster_int.restype = ctypes.c_int
    L.or_ot_theta.argtypes = [i32, i32, dbl]
    L.or_ot_theta.restype = dbl
    L.or_ot_counts.argtypes = [_f64p, _f64p, i32, i32, dbl, _i32p, _i32p]
    L.or_ot_counts.restype = ctypes.c_int
    L.or_ot_fixup.argtypes = [_f64p, i64, i32, i32, _f64p, _f64p, dbl, _i32p, _f64p]
    L.or_ot_fixup.restype = dbl


def theta(nB, nA, eps):
    return float(lib().or_ot_theta(nB, nA, float(eps)))


def counts(nu, mu, eps):
    nu = np.ascontiguousarray(nu, np.float64)
    mu = np.ascontiguousarray(mu, np.float64)
    S = np.empty(nu.size, np.int32)
    D = np.empty(mu.size, np.int32)
    if lib().or_ot_counts(nu, mu, nu.size, mu.size, float(eps), S, D) != OK:
        raise ValueError("bad masses")
    return S, D


def cluster_int(cb, S, D, T, mode=0, cap=None):
    """Cluster phases on integer copy counts S (rows) and D (columns)."""
    cb = np.ascontiguousarray(cb, np.int32)
    nB, nA = cb.shape
    S = np.ascontiguousarray(S, np.int32)
    D = np.ascontiguousarray(D, np.int32)
    out = {k: np.empty(nB, np.int32) for k in ("F", "f")}
    out.update({k: np.empty(nA, np.int32) for k in ("kmin", "clo", "chi")})
    plo = np.empty((nB, nA), np.int32)
    phi = np.empty((nB, nA), np.int32)
    st = Stats()
    rc = lib().or_ot_cluster_int(cb, nB, nA, S, D, int(T), int(mode),
                                 int(cap if cap is not None else 1 << 40), out["F"], out["f"],
                                 out["kmin"], out["clo"], out["chi"], plo, phi, ctypes.byref(st))
    if rc != OK:
        raise RuntimeError(f"oracle OT failed rc={rc}")
    out.update(plan_lo=plo, plan_hi=phi, stats=st.as_dict())
    return out


def ot_phase_cap(eps, S_total):
    K = int(np.floor(1.0 / eps))
    T = int(np.floor(eps * S_total))
    return (S_total * (2 * K + 3)) // (T + 1) + 1


def fixup(C, nu, mu, theta_, cnt):
    """The plan from matched copy counts cnt [nB][nA] and the fix-up alone:
    returns (dense FP64 mass, FP64 cost)."""
    C = np.ascontiguousarray(C, np.float64)
    nB, nA = C.shape
    mass = np.empty((nB, nA), np.float64)
    cost = float(lib().or_ot_fixup(C, nA, nB, nA, np.ascontiguousarray(nu, np.float64),
                                   np.ascontiguousarray(mu, np.float64), float(theta_),
                                   np.ascontiguousarray(cnt, np.int32), mass))
    return mass, cost


def ot(C, nu, mu, eps, mode=0):
    """Whole OT oracle: Sec. 4 scaling, cluster phases, plan, fix-up, cost."""
    C = np.ascontiguousarray(C, np.float64)
    nB, nA = C.shape
    cb = quantise(C, eps)
    S, D = counts(nu, mu, eps)
    S_total = int(S.sum())
    T = int(np.floor(eps * S_total))
    r = cluster_int(cb, S, D, T, mode=mode, cap=ot_phase_cap(eps, S_total))
    th = theta(nB, nA, eps)
    mass = np.empty((nB, nA), np.float64)
    cnt = np.ascontiguousarray(r["plan_lo"] + r["plan_hi"], np.int32)
    cost = float(lib().or_ot_fixup(C, nA, nB, nA, np.ascontiguousarray(nu, np.float64),
                                   np.ascontiguousarray(mu, np.float64), th, cnt, mass))
    r.update(mass=mass, cost=cost, S=S, D=D, T=T, theta=th, cbar=cb, counts=cnt)
    return r
