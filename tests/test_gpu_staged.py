"""GPU tests of pr_assign_staged (a host cost matrix copied to the device in
row chunks, each chunk rounded while the next is copied): its results equal
pr_assign on the same costs in device memory bit for bit (matching, both
dual vectors, phases, rounds, examined entries, cost), and the oracle's on a
small case; ragged last chunks, padded rows, FP32 and 16-bit storage; pinned
and pageable host memory; refused pointers."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2203_03732_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("row_to_col", "col_to_row", "y_row", "y_col")


@pytest.fixture(scope="module")
def prot():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_03732_gb300 import build
    build.build()
    import paper_2203_03732_gb300 as P
    return P


def same_solve(got, ref):
    for k in FIELDS:
        assert np.array_equal(got[k].cpu().numpy(), ref[k].cpu().numpy()), k
    for k in ("phases", "rounds", "cells_examined", "free_at_stop"):
        assert got["stats"][k] == ref["stats"][k], k
    assert float(got["cost"]) == float(ref["cost"].cpu())


@pytest.mark.parametrize("n_rows,n_cols,pad,dtype,eps,pinned", [
    (3000, 3000, 0, np.float64, 0.01, True),     # 24 KB rows: chunks of 1365 rows, the last ragged
    (2500, 3100, 5, np.float64, 0.003, True),    # padded rows, 16-bit storage
    (4100, 4100, 3, np.float32, 0.02, False),    # FP32, pageable host memory
    (1, 7, 0, np.float64, 0.5, True),            # one row
])
def test_staged_equals_device_solve(prot, n_rows, n_cols, pad, dtype, eps, pinned):
    import torch
    C = W.assignment_euclid_2d(n_rows, 5 + n_rows, n_a=n_cols).astype(dtype)
    host = torch.zeros((n_rows, n_cols + pad), dtype=torch.float64 if dtype == np.float64 else torch.float32)
    host[:, :n_cols] = torch.from_numpy(C)
    if pinned:
        host = host.pin_memory()
    Ch = host[:, :n_cols]
    got = prot.assign(Ch, eps)
    ref = prot.assign(Ch.cuda(), eps)
    same_solve(got, ref)


def test_staged_full_size_and_oracle(prot):
    """n = 10,000, eps = 0.01 from pinned host memory (25 chunks) equals the
    device solve; a small case equals the oracle."""
    import torch
    C = W.assignment_euclid_2d(10000, 0)
    Ch = torch.from_numpy(C).pin_memory()
    same_solve(prot.assign(Ch, 0.01), prot.assign(Ch.cuda(), 0.01))
    C = W.assignment_euclid_2d(777, 4)
    got = prot.assign(torch.from_numpy(C).pin_memory(), 0.02)
    ref = oracle.assign(C, 0.02, oracle.MODE_EVICT_RESUME)
    for k in FIELDS:
        assert np.array_equal(got[k].numpy(), ref[k]), k
    assert got["stats"]["phases"] == ref["stats"]["phases"]
    assert abs(float(got["cost"]) - ref["cost"]) <= 1e-12 * ref["cost"]


def test_staged_invalid_cost_reported(prot):
    """A NaN in the last chunk is reported as PR_ERR_INVALID."""
    import torch
    C = W.assignment_euclid_2d(2000, 8)
    C[-1, 3] = np.nan
    with pytest.raises(prot.PrError) as e:
        prot.assign(torch.from_numpy(C).pin_memory(), 0.05)
    assert e.value.status == -1


def test_staged_refuses_wrong_memory(prot):
    """C_host in device memory, or C_dev in host memory, is refused before
    anything is enqueued."""
    import torch
    from paper_2203_03732_gb300 import _lib
    L = _lib.load()
    n = 64
    Cd = torch.rand(n, n, dtype=torch.float64, device="cuda")
    Ch = Cd.cpu().pin_memory()
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4)]
    cost = torch.empty((), dtype=torch.float64, device="cuda")
    ws = torch.empty(L.pr_assign_workspace(n, n), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for src, dst in ((Cd, Cd), (Ch, Ch)):
        rc = L.pr_assign_staged(src.data_ptr(), dst.data_ptr(), _lib.PR_F64, n, n, n, 0.1,
                                *[o.data_ptr() for o in outs], cost.data_ptr(), None,
                                ws.data_ptr(), ws.numel(), stream)
        assert rc == _lib.PR_ERR_INVALID
    rc = L.pr_assign_staged(Ch.data_ptr(), Cd.data_ptr(), _lib.PR_F64, n, n, n, 0.1,
                            *[o.data_ptr() for o in outs], cost.data_ptr(), None,
                            ws.data_ptr(), ws.numel(), stream)
    assert rc == _lib.PR_OK
    torch.cuda.synchronize()
