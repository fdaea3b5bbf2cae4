"""Oracle wrappers for the point-cloud forms (test infrastructure only):
costs from points, one point-cloud solve, the reference gradient."""
from __future__ import annotations

import ctypes

import numpy as np

from . import Stats, lib, OK

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def _declare(L):
    i32, dbl = ctypes.c_int32, ctypes.c_double
    L.or_points_cost.argtypes = [_f32p, _f32p, i32, i32, i32, i32, _f32p]
    L.or_points_cost.restype = None
    L.or_points_match_cost.argtypes = [_f32p, _f32p, i32, i32, i32, _i32p]
    L.or_points_match_cost.restype = dbl
    L.or_assign_points.argtypes = [_f32p, _f32p, i32, i32, i32, i32, dbl, _i32p, _i32p, _i32p,
                                   _i32p, ctypes.POINTER(dbl), ctypes.POINTER(Stats)]
    L.or_assign_points.restype = ctypes.c_int
    L.or_sqeuclid_backward.argtypes = [_f32p, _f32p, i32, i32, _i32p, ctypes.c_float, _f32p, _f32p]
    L.or_sqeuclid_backward.restype = None


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def cost_matrix(XA, XB, squared=True):
    """Normalised FP32 cost matrix C[b, a] (rows = B) from points."""
    XA, XB = _f32(XA), _f32(XB)
    C = np.empty((XB.shape[0], XA.shape[0]), np.float32)
    lib().or_points_cost(XA, XB, XA.shape[0], XB.shape[0], XA.shape[1], int(squared), C)
    return C


def match_cost(XA, XB, row_to_col, squared=True):
    XA, XB = _f32(XA), _f32(XB)
    return float(lib().or_points_match_cost(XA, XB, XB.shape[0], XA.shape[1], int(squared),
                                            np.ascontiguousarray(row_to_col, np.int32)))


def assign_points(XA, XB, eps, squared=True):
    """One point-cloud problem: rows = XB, columns = XA."""
    XA, XB = _f32(XA), _f32(XB)
    nA, nB, d = XA.shape[0], XB.shape[0], XA.shape[1]
    mb = np.empty(nB, np.int32)
    ma = np.empty(nA, np.int32)
    yb = np.empty(nB, np.int32)
    ya = np.empty(nA, np.int32)
    c = ctypes.c_double()
    st = Stats()
    rc = lib().or_assign_points(XA, XB, nA, nB, d, int(squared), float(eps), mb, ma, yb, ya,
                                ctypes.byref(c), ctypes.byref(st))
    if rc != OK:
        raise RuntimeError(f"oracle point solve failed rc={rc}")
    return dict(row_to_col=mb, col_to_row=ma, y_row=yb, y_col=ya, cost=c.value, stats=st.as_dict())


def sqeuclid_backward(X, Y, row_to_col, g):
    """Gradient of (g/n) sum_i |x_i - y_sigma(i)|^2 w.r.t. X (rows) and Y."""
    X, Y = _f32(X), _f32(Y)
    gX = np.empty_like(X)
    gY = np.empty_like(Y)
    lib().or_sqeuclid_backward(X, Y, X.shape[0], X.shape[1],
                               np.ascontiguousarray(row_to_col, np.int32), float(g), gX, gY)
    return gX, gY
