"""GPU tests of the certificate (pr_dual_bound, Lemma 3.1) and of the
delta * n guarantee mode (assign_within: eps = delta / 3, Sec. 1 and 2.1)."""
import numpy as np
import pytest

import oracle
from paper_2203_03732_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prot():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_03732_gb300 import build
    build.build()
    import paper_2203_03732_gb300 as P
    return P


def solve(prot, C, eps):
    import torch
    return prot.assign(torch.from_numpy(C).cuda(), eps)


@pytest.mark.parametrize("n,eps", [(2000, 0.01), (777, 0.1), (10000, 0.01)])
def test_bound_is_the_exact_dual_sum(prot, n, eps):
    """L = eps * (sum y - n_rows): exact integer sums, one FP64 product, one
    FP64 difference for the gap; the same on the host, bit for bit."""
    C = W.assignment_euclid_2d(n, 5)
    r = solve(prot, C, eps)
    b = prot.dual_bound(r, eps)
    ys = int(r["y_row"].cpu().numpy().astype(np.int64).sum() + r["y_col"].cpu().numpy().astype(np.int64).sum())
    L = float(np.float64(eps) * np.float64(ys - n))
    assert float(b["lower_bound"]) == L
    assert float(b["gap_bound"]) == float(np.float64(float(r["cost"])) - np.float64(L))


@pytest.mark.parametrize("n,eps,seed", [(60, 0.1, 0), (250, 0.05, 1), (400, 0.02, 2), (300, 0.005, 3)])
def test_bound_is_below_the_optimum(prot, n, eps, seed):
    """L <= OPT <= cost (exact optimum from the oracle's Hungarian solver), so
    cost - L bounds the true additive error cost - OPT."""
    C = W.assignment_sq_euclid_2d(n, seed)
    r = solve(prot, C, eps)
    b = prot.dual_bound(r, eps)
    opt, _ = oracle.hungarian(C)
    L, cost = float(b["lower_bound"]), float(r["cost"])
    assert L <= opt + 1e-12
    assert opt <= cost + 1e-12
    assert cost - opt <= float(b["gap_bound"]) + 1e-12


def test_bound_from_host_result(prot):
    import torch
    C = W.assignment_euclid_2d(500, 8)
    r = prot.assign(torch.from_numpy(C), 0.05)      # host in, host out
    b = prot.dual_bound(r, 0.05)
    assert not b["lower_bound"].is_cuda
    ys = int(r["y_row"].numpy().astype(np.int64).sum() + r["y_col"].numpy().astype(np.int64).sum())
    assert float(b["lower_bound"]) == float(np.float64(0.05) * np.float64(ys - 500))


@pytest.mark.parametrize("delta", [0.3, 0.06])
@pytest.mark.parametrize("seed", range(4))
def test_assign_within_delta_n(prot, delta, seed):
    """cost <= OPT + delta * n_rows for costs in [0, 1]."""
    n = 300
    C = W.assignment_euclid_2d(n, 20 + seed)
    r = prot.assign_within(__import__("torch").from_numpy(C).cuda(), delta)
    opt, _ = oracle.hungarian(C)
    cost = float(r["cost"])
    assert opt - 1e-12 <= cost <= opt + delta * n + 1e-12
    ref = oracle.assign(C, delta / 3.0)
    assert np.array_equal(r["row_to_col"].cpu().numpy(), ref["row_to_col"])


def test_bad_arguments(prot):
    import ctypes
    import torch
    from paper_2203_03732_gb300 import _lib
    L = _lib.load()
    y = torch.zeros(10, dtype=torch.int32, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    assert L.pr_dual_bound(None, y.data_ptr(), 10, 10, 0.1, None, out.data_ptr(), None) == _lib.PR_ERR_INVALID
    assert L.pr_dual_bound(y.data_ptr(), y.data_ptr(), 11, 10, 0.1, None, out.data_ptr(), None) == _lib.PR_ERR_INVALID
    assert L.pr_dual_bound(y.data_ptr(), y.data_ptr(), 10, 10, 1.5, None, out.data_ptr(), None) == _lib.PR_ERR_INVALID
    assert L.pr_dual_bound(y.data_ptr(), y.data_ptr(), 10, 10, 0.1, None, out.data_ptr(),
                           ctypes.c_void_p(0)) == _lib.PR_OK
    torch.cuda.synchronize()
    assert np.isnan(float(out[1].cpu())) and float(out[0].cpu()) == -1.0  # eps * (0 - 10)
