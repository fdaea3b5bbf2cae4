"""GB300-native push-relabel additive approximation for optimal transport.

Lahn, Raghvendra, Zhang, "A Push-Relabel Based Additive Approximation for
Optimal Transport" (arXiv 2203.03732).  The solver runs in the CUDA library
``libprot.so`` behind the C ABI of ``include/prot.h``; this package is a thin
torch-facing wrapper (device memory, streams, argument marshalling).

    assign(C, eps)  -> matching, integer duals (units of eps), cost
"""
from __future__ import annotations

import ctypes

from . import _lib

__all__ = ["assign", "Workspace", "PrError"]

PrError = _lib.PrError


def _torch():
    import torch
    return torch


class Workspace:
    """A reusable device workspace (grown on demand, 256-byte aligned)."""

    def __init__(self, device=None):
        torch = _torch()
        self.device = torch.device(device if device is not None else "cuda")
        self.buf = None

    def get(self, nbytes: int):
        torch = _torch()
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        assert self.buf.data_ptr() % 256 == 0
        return self.buf


_default_ws = {}


def _workspace(device):
    key = str(device)
    if key not in _default_ws:
        _default_ws[key] = Workspace(device)
    return _default_ws[key]


def _stream_handle(torch, device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def assign(C, eps: float, *, sync: bool = True, ws: Workspace | None = None, out=None):
    """Additive eps-approximate assignment (Sec. 2.2 of the paper).

    C: (n_rows, n_cols) float32/float64 tensor with costs in [0, 1],
       n_rows <= n_cols.  A CUDA tensor is solved in place on its device; a
       CPU tensor is copied to the current CUDA device and the results are
       copied back (the end-to-end path).
    Returns a dict: row_to_col, col_to_row (int32), y_row, y_col (int32 duals
    in units of eps), cost (float64 scalar tensor) and, when sync, stats.
    """
    torch = _torch()
    L = _lib.load()
    host_in = not C.is_cuda
    dev = torch.device("cuda", torch.cuda.current_device()) if host_in else C.device
    if host_in:
        Cd = C.to(dev, non_blocking=True)
    else:
        Cd = C
    if Cd.dim() != 2:
        raise ValueError("C must be 2-D")
    if Cd.stride(1) != 1:
        Cd = Cd.contiguous()
    if Cd.dtype == torch.float64:
        dt = _lib.PR_F64
    elif Cd.dtype == torch.float32:
        dt = _lib.PR_F32
    else:
        raise TypeError("C must be float32 or float64")
    nB, nA = Cd.shape
    need = L.pr_assign_workspace(nB, nA)
    if need == 0:
        raise ValueError("invalid sizes: need 1 <= n_rows <= n_cols <= 2^24")
    wsb = (ws or _workspace(dev)).get(need)
    if out is None:
        out = dict(
            row_to_col=torch.empty(nB, dtype=torch.int32, device=dev),
            col_to_row=torch.empty(nA, dtype=torch.int32, device=dev),
            y_row=torch.empty(nB, dtype=torch.int32, device=dev),
            y_col=torch.empty(nA, dtype=torch.int32, device=dev),
            cost=torch.empty((), dtype=torch.float64, device=dev),
        )
    st = _lib.PrStats()
    rc = L.pr_assign(Cd.data_ptr(), dt, Cd.stride(0), nB, nA, float(eps),
                     out["row_to_col"].data_ptr(), out["col_to_row"].data_ptr(),
                     out["y_row"].data_ptr(), out["y_col"].data_ptr(), out["cost"].data_ptr(),
                     ctypes.byref(st) if sync else None, wsb.data_ptr(), wsb.numel(),
                     _stream_handle(torch, dev))
    _lib.check(rc, "pr_assign")
    res = dict(out)
    if sync:
        res["stats"] = st.as_dict()
    if host_in:
        res = {k: (v.cpu() if hasattr(v, "cpu") else v) for k, v in res.items()}
    return res
