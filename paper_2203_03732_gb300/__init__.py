"""GB300-native push-relabel additive approximation for optimal transport.

Lahn, Raghvendra, Zhang, "A Push-Relabel Based Additive Approximation for
Optimal Transport" (arXiv 2203.03732).  The solver runs in the CUDA library
``libprot.so`` behind the C ABI of ``include/prot.h``; this package is a thin
torch-facing wrapper (device memory, streams, argument marshalling).

    assign(C, eps)                     one problem
    assign_within(C, delta)            one problem, cost <= OPT + delta * n_rows
    assign_points(XA, XB, eps)         one problem with the costs formed from points
    dual_bound(result, eps)            lower bound on OPT from a result's duals
    assign_batched(C, sizes, eps)      many square problems, one launch
    assign_batched_points(XA, XB, sizes, eps)   the same with costs from points
    assignment_loss(X, Y, eps)         differentiable mean matched squared distance
"""
from __future__ import annotations

import ctypes

from . import _lib

__all__ = ["assign", "assign_within", "assign_points", "dual_bound", "assign_batched", "assign_batched_points",
           "assign_backward", "ot",
           "assignment_loss", "AssignLoss", "Workspace", "PrError"]

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


def ws_status(ws: Workspace | None = None):
    """Raise PrError if a solve enqueued on `ws` (default: the current
    device's default workspace) recorded a device-side error; synchronises
    the current stream (pr_ws_status).  For calls made with sync=False."""
    torch = _torch()
    w = ws or _workspace(torch.device("cuda", torch.cuda.current_device()))
    if w.buf is None:
        raise ValueError("ws_status: the workspace holds no solve")
    _lib.check(_lib.load().pr_ws_status(w.buf.data_ptr(), _stream_handle(torch, w.buf.device)), "pr_ws_status")


def assign(C, eps: float, *, sync: bool = True, ws: Workspace | None = None, out=None,
           rule: str = "lowest", results_on_device: bool = False, _within: bool = False):
    """Additive eps-approximate assignment (Sec. 2.2 of the paper).

    C: (n_rows, n_cols) float32/float64 tensor with costs in [0, 1],
       n_rows <= n_cols.  A CUDA tensor is solved in place on its device; a
       CPU tensor (pinned memory for asynchronous copies) is copied to the
       current CUDA device in row chunks, each chunk rounded while the next
       is copied (pr_assign_staged; the other rules copy first), and the
       results are copied back (the end-to-end path).
    Returns a dict: row_to_col, col_to_row (int32), y_row, y_col (int32 duals
    in units of eps), cost (float64 scalar tensor) and, when sync, stats.
    rule: the maximal matching of step (I), "lowest" (lowest-index columns),
    "offset" (seeded start columns per row and phase), "israeli-itai"
    (Israeli and Itai's randomized maximal matching, Sec. 3.2) or
    "sequential" (the sequential greedy of Sec. 3.2, computed without
    rounds); see pr_assign_rule.
    results_on_device: for CPU input, leave the results on the device (no
    copy back, no synchronisation when sync is False).
    """
    torch = _torch()
    L = _lib.load()
    host_in = not C.is_cuda
    dev = torch.device("cuda", torch.cuda.current_device()) if host_in else C.device
    if C.dim() != 2:
        raise ValueError("C must be 2-D")
    staged = host_in and rule == "lowest"
    if staged:
        if C.stride(1) != 1:
            C = C.contiguous()
        Cd = torch.empty_strided(C.shape, C.stride(), dtype=C.dtype, device=dev)
    elif host_in:
        Cd = C.to(dev, non_blocking=True)
    else:
        Cd = C
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
    args = (Cd.data_ptr(), dt, Cd.stride(0), nB, nA, float(eps),
            out["row_to_col"].data_ptr(), out["col_to_row"].data_ptr(),
            out["y_row"].data_ptr(), out["y_col"].data_ptr(), out["cost"].data_ptr(),
            ctypes.byref(st) if sync else None, wsb.data_ptr(), wsb.numel(),
            _stream_handle(torch, dev))
    if _within:  # eps holds delta: pr_assign_within runs the solve with delta / 3
        rc = L.pr_assign_within(*args)
    elif staged:
        rc = L.pr_assign_staged(C.data_ptr(), *args)
    elif rule == "lowest":
        rc = L.pr_assign(*args)
    elif rule == "offset":
        rc = L.pr_assign_rule(_lib.PR_RULE_OFFSET, *args)
    elif rule == "israeli-itai":
        rc = L.pr_assign_rule(_lib.PR_RULE_ISRAELI_ITAI, *args)
    elif rule == "sequential":
        rc = L.pr_assign_rule(_lib.PR_RULE_SEQUENTIAL, *args)
    else:
        raise ValueError("rule must be 'lowest', 'offset', 'israeli-itai' or 'sequential'")
    _lib.check(rc, "pr_assign")
    res = dict(out)
    if sync:
        res["stats"] = st.as_dict()
    if host_in and not results_on_device:
        res = {k: (v.cpu() if hasattr(v, "cpu") else v) for k, v in res.items()}
    return res


def assign_points(XA, XB, eps: float, *, metric: str = "euclidean", sync: bool = True,
                  ws: Workspace | None = None, out=None):
    """`assign` with the costs formed on the device from point sets: XB
    (n_rows, dim) are the rows, XA (n_cols, dim) the columns, FP32.  The
    cost is the distance ("euclidean" or "sqeuclidean") scaled by its largest
    value, rounded by Eq. (1); the returned cost is the matched distance sum
    in input units (FP64).  CPU tensors are copied to the current CUDA device
    and the results back."""
    torch = _torch()
    L = _lib.load()
    host_in = not XB.is_cuda
    dev = torch.device("cuda", torch.cuda.current_device()) if host_in else XB.device
    XBd = XB.to(dev, dtype=torch.float32, non_blocking=True).contiguous()
    XAd = XA.to(dev, dtype=torch.float32, non_blocking=True).contiguous()
    if XBd.dim() != 2 or XAd.dim() != 2 or XBd.shape[1] != XAd.shape[1]:
        raise ValueError("XA, XB must be (n, dim) with the same dim")
    m = {"sqeuclidean": _lib.PR_SQEUCLIDEAN, "euclidean": _lib.PR_EUCLIDEAN}[metric]
    nB, nA, d = XBd.shape[0], XAd.shape[0], XBd.shape[1]
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
    rc = L.pr_assign_points(XAd.data_ptr(), XBd.data_ptr(), d, m, nB, nA, float(eps),
                            out["row_to_col"].data_ptr(), out["col_to_row"].data_ptr(),
                            out["y_row"].data_ptr(), out["y_col"].data_ptr(), out["cost"].data_ptr(),
                            ctypes.byref(st) if sync else None, wsb.data_ptr(), wsb.numel(),
                            _stream_handle(torch, dev))
    _lib.check(rc, "pr_assign_points")
    res = dict(out)
    if sync:
        res["stats"] = st.as_dict()
    if host_in:
        res = {k: (v.cpu() if hasattr(v, "cpu") else v) for k, v in res.items()}
    return res


def dual_bound(result, eps: float):
    """Lemma 3.1's certificate of an `assign` result: a lower bound L on the
    optimal cost from the returned duals, and the bound cost - L on the
    solve's additive error (both FP64 scalar tensors on the result's device;
    for a host result they are copied back).  No optimal solver is needed."""
    torch = _torch()
    L = _lib.load()
    host = not result["y_row"].is_cuda
    dev = torch.device("cuda", torch.cuda.current_device()) if host else result["y_row"].device
    yb = result["y_row"].to(dev, dtype=torch.int32).contiguous()
    ya = result["y_col"].to(dev, dtype=torch.int32).contiguous()
    cost = result["cost"].to(dev, dtype=torch.float64).reshape(())
    out = torch.empty(2, dtype=torch.float64, device=dev)
    rc = L.pr_dual_bound(yb.data_ptr(), ya.data_ptr(), yb.numel(), ya.numel(), float(eps),
                         cost.data_ptr(), out.data_ptr(), _stream_handle(torch, dev))
    _lib.check(rc, "pr_dual_bound")
    if host:
        out = out.cpu()
    return {"lower_bound": out[0], "gap_bound": out[1]}


def assign_within(C, delta: float, **kw):
    """A matching whose cost is within delta * n_rows of the optimum (costs
    in [0, 1]), through pr_assign_within: the main routine with parameter
    eps is a 3 eps approximation (Sec. 2.1, Lemma 3.1), and the library runs
    it with eps = delta / 3 as the paper's introduction does.  The duals are
    in units of that eps.  A CPU tensor is copied to the current device
    first.  Keyword arguments go to `assign` (the lowest-index rule)."""
    torch = _torch()
    if not (0.0 < delta < 3.0):
        raise ValueError("need 0 < delta < 3")
    if kw.get("rule", "lowest") != "lowest":
        raise ValueError("assign_within runs the lowest-index rule")
    kw.pop("rule", None)
    if not C.is_cuda:
        C = C.to(torch.device("cuda", torch.cuda.current_device()))
    return assign(C, delta, _within=True, **kw)


def _tune_cache_path():
    import os
    return os.environ.get("PROT_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "prot", "batched_tune.json"))


def _tune_key(torch, dev, kind, sizes, eps, extra=""):
    import numpy as np
    n = np.asarray(sizes, dtype=np.int64)
    name = torch.cuda.get_device_name(dev)
    return f"{name}|{kind}{extra}|P={n.size}|nmax={int(n.max())}|n2={int((n * n).sum())}|eps={eps!r}"


def _tune_lookup(key):
    import json
    try:
        with open(_tune_cache_path()) as f:
            v = json.load(f).get(key)
        return (int(v[0]), int(v[1])) if v else None
    except (OSError, ValueError):
        return None


def _tune_store(key, tune):
    import json
    import os
    path = _tune_cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        try:
            with open(path) as f:
                d = json.load(f)
        except (OSError, ValueError):
            d = {}
        d[key] = [int(tune[0]), int(tune[1])]
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home: the choice is simply not remembered


def _autotune(torch, L, dev, kind, args_src, sizes, n_ptr, eps, out, wsb):
    """Run the library's autotuner for this batch; returns (threads, ctas_per_sm)."""
    best = _lib.PrBatchedTune()
    ms = ctypes.c_float()
    XA, XB, dim, metric, C, dt = args_src
    rc = L.pr_assign_batched_autotune(XA, XB, dim, metric, C, dt, len(sizes), n_ptr, float(eps),
                                      out["row_to_col"].data_ptr(), out["col_to_row"].data_ptr(),
                                      out["y_row"].data_ptr(), out["y_col"].data_ptr(),
                                      out["costs"].data_ptr(), out["phases"].data_ptr(),
                                      ctypes.byref(best), ctypes.byref(ms), wsb.data_ptr(), wsb.numel(),
                                      _stream_handle(torch, dev))
    _lib.check(rc, "pr_assign_batched_autotune")
    return (best.threads, best.ctas_per_sm)


def _tune_struct(tune):
    if tune is None:
        return None
    t = _lib.PrBatchedTune()
    t.threads, t.ctas_per_sm = int(tune[0]), int(tune[1])
    return ctypes.byref(t)


def _batched_outputs(torch, dev, sizes):
    import numpy as np
    tot = int(np.sum(sizes))
    P = len(sizes)
    return dict(
        row_to_col=torch.empty(tot, dtype=torch.int32, device=dev),
        col_to_row=torch.empty(tot, dtype=torch.int32, device=dev),
        y_row=torch.empty(tot, dtype=torch.int32, device=dev),
        y_col=torch.empty(tot, dtype=torch.int32, device=dev),
        costs=torch.empty(P, dtype=torch.float64, device=dev),
        phases=torch.empty(P, dtype=torch.int64, device=dev),
    )


def _sizes_arg(sizes):
    import numpy as np
    n = np.ascontiguousarray(np.asarray(sizes), dtype=np.int32)
    return n, n.ctypes.data_as(ctypes.c_void_p)


def assign_batched(C, sizes, eps: float, *, tune=None, sync: bool = True,
                   ws: Workspace | None = None, out=None):
    """Many independent square problems in one persistent launch.

    C: 1-D CUDA tensor (float32/float64) holding the problems' n_i x n_i cost
    matrices back to back (rows = proposing side), costs in [0, 1].
    sizes: the n_i (host).  Returns packed row_to_col, col_to_row, y_row,
    y_col (offset sum_{j<i} n_j, indices local to each problem), costs[P],
    phases[P] and, when sync, stats (totals).
    """
    torch = _torch()
    L = _lib.load()
    if not C.is_cuda:
        raise ValueError("C must be a CUDA tensor")
    C = C.contiguous()
    dt = {torch.float64: _lib.PR_F64, torch.float32: _lib.PR_F32}.get(C.dtype)
    if dt is None:
        raise TypeError("C must be float32 or float64")
    n, n_ptr = _sizes_arg(sizes)
    if C.numel() != int((n.astype("int64") ** 2).sum()):
        raise ValueError("C does not hold sum n_i^2 elements")
    dev = C.device
    need = L.pr_assign_batched_workspace(len(n), n_ptr)
    if need == 0:
        raise PrError(_lib.PR_ERR_INVALID, "invalid problem sizes (need 1 <= n_i <= 5000)")
    wsb = (ws or _workspace(dev)).get(need)
    out = out or _batched_outputs(torch, dev, n)
    if isinstance(tune, str):
        key = _tune_key(torch, dev, "matrix", n, eps, extra=str(C.dtype))
        tune = _tune_lookup(key)
        if tune is None:
            tune = _autotune(torch, L, dev, "matrix", (None, None, 0, 0, C.data_ptr(), dt), n, n_ptr, eps,
                             out, wsb)
            _tune_store(key, tune)
    st = _lib.PrStats()
    rc = L.pr_assign_batched(C.data_ptr(), dt, len(n), n_ptr, float(eps),
                             out["row_to_col"].data_ptr(), out["col_to_row"].data_ptr(),
                             out["y_row"].data_ptr(), out["y_col"].data_ptr(), out["costs"].data_ptr(),
                             out["phases"].data_ptr(), _tune_struct(tune),
                             ctypes.byref(st) if sync else None, wsb.data_ptr(), wsb.numel(),
                             _stream_handle(torch, dev))
    _lib.check(rc, "pr_assign_batched")
    res = dict(out)
    if sync:
        res["stats"] = st.as_dict()
    return res


def assign_batched_points(XA, XB, sizes, eps: float, *, metric: str = "sqeuclidean", tune=None,
                          sync: bool = True, ws: Workspace | None = None, out=None):
    """Batched solve with costs formed from point sets.

    XA, XB: (sum n_i, dim) float32 CUDA tensors; problem i owns rows
    sum_{j<i} n_j .. + n_i of each; XB are the proposing rows (B), XA the
    columns (A).  metric: "sqeuclidean" or "euclidean".  Costs are scaled per
    problem so the largest is 1; reported costs are in input units.
    """
    torch = _torch()
    L = _lib.load()
    if not (XA.is_cuda and XB.is_cuda):
        raise ValueError("points must be CUDA tensors")
    if XA.dtype != torch.float32 or XB.dtype != torch.float32:
        raise TypeError("points must be float32")
    XA, XB = XA.contiguous(), XB.contiguous()
    if XA.shape != XB.shape or XA.dim() != 2:
        raise ValueError("XA and XB must both be (sum n_i, dim)")
    m = {"sqeuclidean": _lib.PR_SQEUCLIDEAN, "euclidean": _lib.PR_EUCLIDEAN}[metric]
    n, n_ptr = _sizes_arg(sizes)
    if XA.shape[0] != int(n.sum()):
        raise ValueError("points do not hold sum n_i rows")
    dev = XA.device
    need = L.pr_assign_batched_workspace(len(n), n_ptr)
    if need == 0:
        raise PrError(_lib.PR_ERR_INVALID, "invalid problem sizes (need 1 <= n_i <= 5000)")
    wsb = (ws or _workspace(dev)).get(need)
    out = out or _batched_outputs(torch, dev, n)
    if isinstance(tune, str):
        key = _tune_key(torch, dev, "points", n, eps, extra=f"{metric}d{XA.shape[1]}")
        tune = _tune_lookup(key)
        if tune is None:
            tune = _autotune(torch, L, dev, "points", (XA.data_ptr(), XB.data_ptr(), XA.shape[1], m, None, 0),
                             n, n_ptr, eps, out, wsb)
            _tune_store(key, tune)
    st = _lib.PrStats()
    rc = L.pr_assign_batched_points(XA.data_ptr(), XB.data_ptr(), XA.shape[1], m, len(n), n_ptr,
                                    float(eps), out["row_to_col"].data_ptr(),
                                    out["col_to_row"].data_ptr(), out["y_row"].data_ptr(),
                                    out["y_col"].data_ptr(), out["costs"].data_ptr(),
                                    out["phases"].data_ptr(), _tune_struct(tune),
                                    ctypes.byref(st) if sync else None, wsb.data_ptr(), wsb.numel(),
                                    _stream_handle(torch, dev))
    _lib.check(rc, "pr_assign_batched_points")
    res = dict(out)
    if sync:
        res["stats"] = st.as_dict()
    return res


def assign_backward(row_to_col, X, Y, grad_cost, *, grad_C: bool = False):
    """Gradients of L_p = (1/n) sum_i |x_i - y_sigma(i)|^2 for (batch, n, dim)
    FP32 CUDA tensors X (rows) and Y (columns), plans row_to_col (batch*n) and
    incoming gradients grad_cost (batch,).  Returns (grad_X, grad_Y[, grad_C])."""
    torch = _torch()
    L = _lib.load()
    B, n, d = X.shape
    X, Y = X.contiguous(), Y.contiguous()
    g = grad_cost.contiguous().to(torch.float32)
    r2c = row_to_col.contiguous()
    gX = torch.empty_like(X)
    gY = torch.empty_like(Y)
    gC = torch.empty((B, n, n), dtype=torch.float32, device=X.device) if grad_C else None
    rc = L.pr_assign_backward(r2c.data_ptr(), X.data_ptr(), Y.data_ptr(), B, n, d, g.data_ptr(),
                              gX.data_ptr(), gY.data_ptr(), gC.data_ptr() if grad_C else None,
                              _stream_handle(torch, X.device))
    _lib.check(rc, "pr_assign_backward")
    return (gX, gY, gC) if grad_C else (gX, gY)


def _assign_loss_function():
    torch = _torch()

    class AssignLoss(torch.autograd.Function):
        """Mean matched squared distance of point-cloud pairs.

        forward: the batched solver (costs |x - y|^2 scaled per pair so the
        largest is 1, Eq. 1 rounding, Sec. 2.2 phases) gives a plan sigma per
        pair; the loss is (1/n) sum_i |x_i - y_sigma(i)|^2 in input units.
        backward: the hand-written CUDA kernel with the plans held fixed.
        """

        @staticmethod
        def forward(ctx, X, Y, eps):
            B, n, d = X.shape
            sizes = [n] * B
            res = assign_batched_points(Y.detach().reshape(B * n, d), X.detach().reshape(B * n, d),
                                        sizes, eps, metric="sqeuclidean", sync=False, tune="auto")
            ctx.save_for_backward(X, Y, res["row_to_col"])
            ctx.plan = res
            return (res["costs"] / n).to(X.dtype)

        @staticmethod
        def backward(ctx, g):
            X, Y, r2c = ctx.saved_tensors
            gX, gY = assign_backward(r2c, X.detach(), Y.detach(), g)
            return gX, gY, None

    return AssignLoss


_AssignLoss = None


def __getattr__(name):
    global _AssignLoss
    if name == "AssignLoss":
        if _AssignLoss is None:
            _AssignLoss = _assign_loss_function()
        return _AssignLoss
    raise AttributeError(name)


def assignment_loss(X, Y, eps: float):
    """Differentiable (batch,) loss for (batch, n, dim) FP32 CUDA point clouds."""
    return __getattr__("AssignLoss").apply(X, Y, eps)


def ot(C, supply, demand, eps: float, *, plan_cap: int | None = None, ws: Workspace | None = None,
       sync: bool = True):
    """Additive eps-approximate optimal transport (Sec. 4 of the paper).

    C: (n_sup, n_dem) float32/float64 CUDA tensor of costs in [0, 1] (rows =
    supplies); supply, demand: FP64 CUDA tensors of masses summing to 1.
    Returns dict(plan_row, plan_col, plan_mass (the nnz plan triples), cost,
    y_sup, dem_kmin, dem_lo, dem_hi (cluster duals, units of eps), stats).
    sync=False enqueues the solve and returns at once: the plan arrays are
    then returned at their full capacity with plan_nnz on the device, no
    stats, and device errors are read later with ws_status(ws)."""
    torch = _torch()
    L = _lib.load()
    if not (C.is_cuda and supply.is_cuda and demand.is_cuda):
        raise ValueError("C, supply and demand must be CUDA tensors")
    if C.stride(1) != 1:
        C = C.contiguous()
    dt = {torch.float64: _lib.PR_F64, torch.float32: _lib.PR_F32}.get(C.dtype)
    if dt is None:
        raise TypeError("C must be float32 or float64")
    nB, nA = C.shape
    supply = supply.contiguous().to(torch.float64)
    demand = demand.contiguous().to(torch.float64)
    dev = C.device
    need = L.pr_ot_workspace(nB, nA)
    if need == 0:
        raise PrError(_lib.PR_ERR_INVALID, "invalid sizes")
    wsb = (ws or _workspace(dev)).get(need)
    n = max(nB, nA)
    if plan_cap is None:
        # matched pairs are at most the supply copies (<= theta) and nB*nA;
        # the fix-up adds at most nB + nA pairs
        plan_cap = int(min(nB * nA, 4 * n / eps + 1) + nB + nA)
    i32 = dict(dtype=torch.int32, device=dev)
    out = dict(plan_row=torch.empty(plan_cap, **i32), plan_col=torch.empty(plan_cap, **i32),
               plan_mass=torch.empty(plan_cap, dtype=torch.float64, device=dev),
               plan_nnz=torch.zeros((), dtype=torch.int64, device=dev),
               y_sup=torch.empty(nB, **i32), dem_kmin=torch.empty(nA, **i32),
               dem_lo=torch.empty(nA, **i32), dem_hi=torch.empty(nA, **i32),
               cost=torch.empty((), dtype=torch.float64, device=dev))
    st = _lib.PrStats()
    rc = L.pr_ot(C.data_ptr(), dt, C.stride(0), nB, nA, supply.data_ptr(), demand.data_ptr(),
                 float(eps), plan_cap, out["plan_row"].data_ptr(), out["plan_col"].data_ptr(),
                 out["plan_mass"].data_ptr(), out["plan_nnz"].data_ptr(), out["y_sup"].data_ptr(),
                 out["dem_kmin"].data_ptr(), out["dem_lo"].data_ptr(), out["dem_hi"].data_ptr(),
                 out["cost"].data_ptr(), ctypes.byref(st) if sync else None, wsb.data_ptr(), wsb.numel(),
                 _stream_handle(torch, dev))
    _lib.check(rc, "pr_ot")
    if not sync:
        return out
    nnz = int(out["plan_nnz"].item())
    for k in ("plan_row", "plan_col", "plan_mass"):
        out[k] = out[k][:nnz]
    out["stats"] = st.as_dict()
    return out
