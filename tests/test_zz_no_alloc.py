"""pr_assign_noalloc: the allocation-free form of pr_assign.

Some callers cannot allocate device memory (while a stream is captured into
a CUDA graph, inside an application that forbids device allocations after
start-up, or in a loop that must not enter the allocator).  This entry point
takes no workspace: it uses one fixed-size device array inside the library.
The test calls it through the C ABI and checks it against pr_assign (with a
caller workspace) on two calls in a row: the matching, both dual vectors and
the counters bit for bit, the FP64 cost within 1e-12 relative.  Each case is
also checked against the CPU oracle on the same input, so the comparison
does not rest on the CUDA path alone, and one case runs with 16-bit rounded
costs (floor(1/eps) > 252).  The cost matrix may sit in pinned host memory
(read through its device mapping); pageable host memory is refused before
any kernel runs.  It lives in its own file, collected last, and works alone
in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

from paper_2203_03732_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_03732_gb300 import build
    build.build()
    from paper_2203_03732_gb300 import _lib
    return _lib


def call_noalloc(_lib, C, eps):
    import torch
    L = _lib.load()
    nB, nA = C.shape
    i32 = dict(dtype=torch.int32, device="cuda")
    out = dict(row_to_col=torch.empty(nB, **i32), col_to_row=torch.empty(nA, **i32),
               y_row=torch.empty(nB, **i32), y_col=torch.empty(nA, **i32),
               cost=torch.empty((), dtype=torch.float64, device="cuda"))
    st = _lib.PrStats()
    dt = _lib.PR_F64 if C.dtype == torch.float64 else _lib.PR_F32
    rc = L.pr_assign_noalloc(C.data_ptr(), dt, C.stride(0), nB, nA, float(eps),
                             out["row_to_col"].data_ptr(), out["col_to_row"].data_ptr(),
                             out["y_row"].data_ptr(), out["y_col"].data_ptr(), out["cost"].data_ptr(),
                             ctypes.byref(st),
                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(rc, "pr_assign_noalloc")
    return out, st.as_dict()


def call_with_workspace(C, eps):
    import paper_2203_03732_gb300 as P
    r = P.assign(C, eps)
    return r, r["stats"]


def same(a, sa, b, sb):
    import torch
    for k in ("row_to_col", "col_to_row", "y_row", "y_col"):
        assert torch.equal(a[k], b[k]), k
    for k in ("phases", "rounds", "free_at_stop", "threshold"):
        assert sa[k] == sb[k], k
    ca, cb = float(a["cost"].cpu()), float(b["cost"].cpu())
    assert abs(ca - cb) <= 1e-12 * max(abs(cb), 1e-300)


def same_as_oracle(got, sgot, ref):
    for k in ("row_to_col", "col_to_row", "y_row", "y_col"):
        assert np.array_equal(got[k].cpu().numpy(), ref[k]), k
    assert sgot["phases"] == ref["stats"]["phases"]
    assert sgot["rounds"] == ref["stats"]["rounds"]
    c = float(got["cost"].cpu())
    assert abs(c - ref["cost"]) <= 1e-12 * max(abs(ref["cost"]), 1e-300)


# (1024, 1024) at eps = 0.003 has floor(1/eps) = 333 > 252: 16-bit rounded costs
@pytest.mark.parametrize("shape,eps,dtype", [((1024, 1024), 0.01, "f64"), ((300, 517), 0.1, "f32"),
                                             ((1024, 1024), 0.003, "f64")])
def test_noalloc_matches_pr_assign_twice(lib, shape, eps, dtype):
    import torch
    import oracle
    nB, nA = shape
    C = W.assignment_euclid_2d(nB, 7, n_a=nA)
    Cn = C if dtype == "f64" else C.astype(np.float32)
    Ct = torch.from_numpy(Cn).cuda()
    ref, sref = call_with_workspace(Ct, eps)
    want = oracle.assign(Cn, eps)
    for _ in range(2):  # the second call starts from the first call's leftovers
        got, sgot = call_noalloc(lib, Ct, eps)
        same(got, sgot, ref, sref)
        same_as_oracle(got, sgot, want)


def test_noalloc_reads_pinned_host_costs_and_refuses_pageable(lib):
    import torch
    C = W.assignment_euclid_2d(200, 3, n_a=260)
    dev = torch.from_numpy(C).cuda()
    ref, sref = call_with_workspace(dev, 0.05)
    pinned = torch.from_numpy(C).pin_memory()
    got, sgot = call_noalloc(lib, pinned, 0.05)
    same(got, sgot, ref, sref)
    pageable = torch.from_numpy(C.copy())
    with pytest.raises(lib.PrError) as e:
        call_noalloc(lib, pageable, 0.05)
    assert e.value.status == lib.PR_ERR_INVALID


def test_noalloc_rejects_sizes_beyond_its_limit(lib):
    import torch
    C = torch.rand(8, 1025, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.PrError) as e:
        call_noalloc(lib, C, 0.1)
    assert e.value.status == lib.PR_ERR_INVALID
    assert "1024" in str(e.value)
