"""GPU parity of pr_assign against the CPU oracle (bit-exact matching, both
dual vectors and the phase/round counts; FP64 cost within 1e-12 relative).

Sizes span one chunk, several chunks and ragged tails of the row scan
(1536-column byte chunks, 768-column 16-bit chunks, 8- and 16-column vectors), the unbalanced case, FP32 input,
closed-form special cases, and the full n = 10,000 workloads.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_2203_03732_gb300 import workloads as W

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-12


@pytest.fixture(scope="module")
def prot():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_03732_gb300 import build
    build.build()
    import paper_2203_03732_gb300 as P
    return P


def gpu_solve(P, C, eps):
    import torch
    r = P.assign(torch.from_numpy(C).cuda(), eps)
    out = {k: r[k].cpu().numpy() for k in ("row_to_col", "col_to_row", "y_row", "y_col")}
    out["cost"] = float(r["cost"].cpu())
    out["stats"] = r["stats"]
    return out


def assert_parity(got, ref):
    for k in ("row_to_col", "col_to_row", "y_row", "y_col"):
        assert np.array_equal(got[k], ref[k]), f"{k} differs"
    assert got["stats"]["phases"] == ref["stats"]["phases"]
    assert got["stats"]["rounds"] == ref["stats"]["rounds"]
    assert got["stats"]["free_at_stop"] == ref["stats"]["free_at_stop"]
    assert got["stats"]["threshold"] == ref["threshold"]
    assert abs(got["cost"] - ref["cost"]) <= COST_RTOL * max(abs(ref["cost"]), 1e-300)


@pytest.mark.parametrize("seed", range(30))
def test_config_n1000_sq_euclid(prot, seed):
    C = W.assignment_sq_euclid_2d(1000, seed)
    assert_parity(gpu_solve(prot, C, 0.1), oracle.assign(C, 0.1))


@pytest.mark.parametrize("n", [7, 64, 257, 1000, 2049, 4097, 5003])
@pytest.mark.parametrize("eps", [0.1, 0.01, 0.005])
def test_sizes_and_eps(prot, n, eps):
    C = W.assignment_euclid_2d(n, 11 + n)
    assert_parity(gpu_solve(prot, C, eps), oracle.assign(C, eps))


@pytest.mark.parametrize("nB,nA", [(100, 173), (1000, 4100), (1, 9), (33, 8200)])
def test_unbalanced(prot, nB, nA):
    C = W.assignment_euclid_2d(nB, 3, n_a=nA)
    for eps in (0.1, 0.02):
        assert_parity(gpu_solve(prot, C, eps), oracle.assign(C, eps))


def test_float32_input(prot):
    C = W.assignment_euclid_2d(1500, 4).astype(np.float32)
    assert_parity(gpu_solve(prot, C, 0.01), oracle.assign(C, 0.01))


def test_leading_dimension(prot):
    import torch
    C = W.assignment_euclid_2d(600, 5)
    big = np.zeros((600, 640))
    big[:, :600] = C
    Ct = torch.from_numpy(big).cuda()[:, :600]
    assert Ct.stride(0) == 640
    r = prot.assign(Ct, 0.01)
    ref = oracle.assign(C, 0.01)
    assert np.array_equal(r["row_to_col"].cpu().numpy(), ref["row_to_col"])
    assert np.array_equal(r["y_row"].cpu().numpy(), ref["y_row"])


@pytest.mark.parametrize("n,k,eps", [(300, 0.55, 0.1), (129, 1.0, 0.25), (1, 0.73, 0.001)])
def test_constant_costs(prot, n, k, eps):
    C = np.full((n, n), k)
    got, ref = gpu_solve(prot, C, eps), oracle.assign(C, eps)
    assert_parity(got, ref)
    assert got["row_to_col"].tolist() == list(range(n))


def test_zero_diagonal_and_permutation(prot):
    n = 4500
    C = 1.0 - np.eye(n)
    got = gpu_solve(prot, C, 0.1)
    assert got["row_to_col"].tolist() == list(range(n))
    assert got["stats"]["phases"] == 1 and got["stats"]["rounds"] == 1
    pi = np.random.default_rng(0).permutation(n)
    C = np.ones((n, n))
    C[np.arange(n), pi] = 0.0
    got = gpu_solve(prot, C, 0.2)
    assert got["row_to_col"].tolist() == pi.tolist()


def test_smallest_eps(prot):
    """floor(1/eps) = 32766, the largest the 16-bit keys allow."""
    eps = 1.0 / 32766.5
    C = W.assignment_euclid_2d(40, 9)
    assert_parity(gpu_solve(prot, C, eps), oracle.assign(C, eps))


@pytest.mark.parametrize("eps", [0.1, 0.01, 0.005])
def test_full_size_n10000(prot, eps):
    """The n = 10,000 Euclidean workload in the launch configuration the
    bench times, compared in full with the oracle."""
    C = W.assignment_euclid_2d(10000, 0)
    assert_parity(gpu_solve(prot, C, eps), oracle.assign(C, eps))


def dual_certificate(C, eps, got):
    """Lemma 3.1 on the GPU's own duals, a check that needs no optimum:
    Eq. (2) and (3) hold on every edge (in units of eps) for the matching
    before completion, and c(M) <= L + 2 eps n_B + T with
    L = eps (sum y - n_B) a lower bound on OPT."""
    nB = C.shape[0]
    yb = got["y_row"].astype(np.int64)
    ya = got["y_col"].astype(np.int64)
    assert yb.min() >= 1 and ya.max() <= 0
    T = oracle.threshold(eps, nB)
    for r0 in range(0, nB, 1000):  # row blocks keep the host memory small
        cb = oracle.quantise(C[r0:r0 + 1000], eps).astype(np.int64)
        s = cb + 1 - yb[r0:r0 + 1000, None] - ya[None, :]
        assert s.min() >= 0                                   # Eq. (2)
        m = got["row_to_col"][r0:r0 + 1000]
        tight = s[np.arange(len(m)), m] == 1                  # Eq. (3)
        assert (~tight).sum() <= T  # only completion edges may break it
    L = eps * (yb.sum() + ya.sum() - nB)
    assert got["cost"] <= L + 2 * eps * nB + T + 1e-6


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_full_size_n10000_more_seeds(prot, seed):
    """Five more seeds of the n = 10,000 workload at eps = 0.01: parity in
    full, and the dual certificate on the GPU's duals."""
    C = W.assignment_euclid_2d(10000, seed)
    got = gpu_solve(prot, C, 0.01)
    assert_parity(got, oracle.assign(C, 0.01))
    dual_certificate(C, 0.01, got)


FORMS = ["grid", "grid-slots", "cluster"]


def set_form(monkeypatch, form):
    """grid: whole grid, rows scanned from registers; grid-slots: whole grid,
    CTAs with many rows scan them from bulk-copied shared-memory slots;
    cluster: one thread-block cluster."""
    monkeypatch.setenv("PR_PHASE_MODE", "cluster" if form == "cluster" else "grid")
    monkeypatch.setenv("PR_SCAN", "auto" if form == "grid-slots" else "regs")


def assert_cells(got, C, eps):
    """The scans examine exactly the entries the oracle's evict-resume mode
    examines (an evicted row starts after the column it lost), and that mode
    gives the same result as the plain one."""
    ref = oracle.assign(C, eps, mode=oracle.MODE_EVICT_RESUME)
    assert_parity(got, ref)
    assert got["stats"]["cells_examined"] == ref["stats"]["scanned"]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,eps", [(64, 0.1), (1000, 0.01), (4097, 0.005), (5003, 0.1), (700, 0.002)])
def test_all_phase_loop_forms(prot, monkeypatch, form, n, eps):
    """The phase loop on the whole grid (barriers through L2; rows scanned
    from registers or from bulk-copied shared-memory slots) and in one
    thread-block cluster (barriers through distributed shared memory) give
    the same bit-exact result, in byte and in 16-bit storage."""
    set_form(monkeypatch, form)
    C = W.assignment_euclid_2d(n, 41 + n)
    got = gpu_solve(prot, C, eps)
    assert_parity(got, oracle.assign(C, eps))
    assert_cells(got, C, eps)
    assert got["stats"]["loop_cluster"] == (1 if form == "cluster" else 0)
    assert got["stats"]["loop_ctas"] >= (8 if form == "cluster" else 100)


@pytest.mark.parametrize("form", FORMS)
def test_full_size_n10000_all_forms(prot, monkeypatch, form):
    set_form(monkeypatch, form)
    C = W.assignment_euclid_2d(10000, 0)
    got = gpu_solve(prot, C, 0.01)
    assert_cells(got, C, 0.01)
    assert got["stats"]["loop_cluster"] == (1 if form == "cluster" else 0)


def test_repeat_is_deterministic(prot):
    C = W.assignment_euclid_2d(3000, 21)
    a = gpu_solve(prot, C, 0.01)
    b = gpu_solve(prot, C, 0.01)
    for k in ("row_to_col", "y_row", "y_col"):
        assert np.array_equal(a[k], b[k])
    assert a["cost"] == b["cost"]


# ---------------------------------------------------------------------------
# Error paths (host-side checks and device-side status; nothing faults)
# ---------------------------------------------------------------------------

def test_cost_out_of_range_reported(prot):
    import torch
    C = W.assignment_euclid_2d(100, 1)
    C[37, 5] = 1.5
    with pytest.raises(prot.PrError) as e:
        prot.assign(torch.from_numpy(C).cuda(), 0.1)
    assert e.value.status == -1
    C[37, 5] = np.nan
    with pytest.raises(prot.PrError):
        prot.assign(torch.from_numpy(C).cuda(), 0.1)


def test_bad_arguments(prot):
    import torch
    from paper_2203_03732_gb300 import _lib
    L = _lib.load()
    C = torch.rand(10, 20, dtype=torch.float64, device="cuda")
    for eps in (0.0, 1.0, -0.1, 1e-6):
        with pytest.raises(prot.PrError):
            prot.assign(C, eps)
    with pytest.raises(ValueError):
        prot.assign(C.t().contiguous(), 0.1)  # n_rows > n_cols
    # workspace too small / misaligned
    out = [torch.empty(10, dtype=torch.int32, device="cuda") for _ in range(2)]
    outa = [torch.empty(20, dtype=torch.int32, device="cuda") for _ in range(2)]
    cost = torch.empty((), dtype=torch.float64, device="cuda")
    ws = torch.empty(L.pr_assign_workspace(10, 20), dtype=torch.uint8, device="cuda")
    st = _lib.PrStats()
    rc = L.pr_assign(C.data_ptr(), 1, 20, 10, 20, 0.1, out[0].data_ptr(), outa[0].data_ptr(),
                     out[1].data_ptr(), outa[1].data_ptr(), cost.data_ptr(), ctypes.byref(st),
                     ws.data_ptr(), ws.numel() - 1, None)
    assert rc == _lib.PR_ERR_WORKSPACE
    rc = L.pr_assign(C.data_ptr(), 1, 20, 10, 20, 0.1, out[0].data_ptr(), outa[0].data_ptr(),
                     out[1].data_ptr(), outa[1].data_ptr(), cost.data_ptr(), ctypes.byref(st),
                     ws.data_ptr() + 8, ws.numel() - 8, None)
    assert rc == _lib.PR_ERR_WORKSPACE
    rc = L.pr_assign(C.data_ptr(), 1, 19, 10, 20, 0.1, out[0].data_ptr(), outa[0].data_ptr(),
                     out[1].data_ptr(), outa[1].data_ptr(), cost.data_ptr(), ctypes.byref(st),
                     ws.data_ptr(), ws.numel(), None)
    assert rc == _lib.PR_ERR_INVALID
    assert b"ldc" in L.pr_last_error()


@pytest.mark.parametrize("form", FORMS)
def test_barrier_timeout_reported_not_hung(prot, monkeypatch, form):
    """A one-cycle spin budget makes every waiting CTA give up at its first
    barrier (grid or cluster form): the call returns PR_ERR_TIMEOUT and the
    context stays usable (the next solve is exact)."""
    import torch
    set_form(monkeypatch, form)
    C = W.assignment_euclid_2d(2000, 2)
    monkeypatch.setenv("PR_SPIN_LIMIT_CYCLES", "1")
    with pytest.raises(prot.PrError) as e:
        prot.assign(torch.from_numpy(C).cuda(), 0.01)
    assert e.value.status == -3
    monkeypatch.delenv("PR_SPIN_LIMIT_CYCLES")
    assert_parity(gpu_solve(prot, C, 0.01), oracle.assign(C, 0.01))


def test_async_status_query(prot):
    import torch
    from paper_2203_03732_gb300 import _lib
    C = W.assignment_euclid_2d(200, 1)
    C[3, 3] = -0.5
    ws = prot.Workspace("cuda")
    with pytest.raises(prot.PrError):
        prot.assign(torch.from_numpy(C).cuda(), 0.1, ws=ws)
    C[3, 3] = 0.5
    r = prot.assign(torch.from_numpy(C).cuda(), 0.1, ws=ws, sync=False)
    rc = _lib.load().pr_ws_status(ctypes.c_void_p(ws.buf.data_ptr()), None)
    assert rc == 0
    ref = oracle.assign(C, 0.1)
    assert np.array_equal(r["row_to_col"].cpu().numpy(), ref["row_to_col"])


@pytest.mark.parametrize("eps,dtype", [(0.1, np.float64), (0.01, np.float64), (1.0 / 3.0, np.float64),
                                       (0.005, np.float32), (1.0 / 32766.5, np.float64)])
def test_rounding_on_and_next_to_multiples_of_eps(prot, eps, dtype):
    """Costs on multiples of eps and one ulp either side, plus 0, -0.0, 1 and
    denormals: Eq. (1)'s exact floor decides every one of them, so any
    rounding slip changes the duals."""
    g = np.random.default_rng(3)
    n = 384
    K = int(np.floor(1.0 / eps))
    k = g.integers(0, K + 1, size=(n, n)).astype(dtype)
    base = (k * dtype(eps)).astype(dtype)
    side = g.integers(-1, 2, size=(n, n))
    C = np.where(side < 0, np.nextafter(base, dtype(0)), np.where(side > 0, np.nextafter(base, dtype(2)), base))
    C = np.clip(C, 0, 1).astype(dtype)
    C[0, :4] = [0.0, -0.0, 1.0, np.finfo(dtype).tiny / 4]
    assert_parity(gpu_solve(prot, C, eps), oracle.assign(C, eps))


@pytest.mark.parametrize("K", [125, 126, 252, 253])
def test_byte_test_forms_at_their_limits(prot, K):
    """floor(1/eps) = 125 is the largest for the plain-add byte pre-test,
    126 .. 252 take the carry-isolated one, 253 switches to 16-bit storage:
    parity and the exact examined-entry count on either side of each limit."""
    eps = 1.0 / (K + 0.5)
    C = W.assignment_euclid_2d(1500, 60 + K)
    got = gpu_solve(prot, C, eps)
    assert_parity(got, oracle.assign(C, eps))
    assert_cells(got, C, eps)


@pytest.mark.parametrize("eps", [0.75, 0.5, 0.25, 0.1])
def test_mnist_shaped_workload(prot, eps):
    """The paper's second experiment on seeded MNIST-shaped images (the
    dataset is not available): unit-mass 28x28 images, L1 cost / max, the
    paper's eps values; parity with the oracle and the Lemma 3.1 bound
    against the exact optimum."""
    A, B = W.mnist_shaped_pair(500, 11)
    C = W.l1_cost(A, B)
    got = gpu_solve(prot, C, eps)
    ref = oracle.assign(C, eps)
    assert_parity(got, ref)
    opt, _ = oracle.hungarian(C)
    assert opt - 1e-9 <= got["cost"] <= opt + 3 * eps * 500 + 1e-9


def test_widest_problem_the_key_copy_holds(prot):
    """n_cols at the limit the library reports (the shared-memory copy of the
    column keys and the taken set): parity with the oracle there, and
    PR_ERR_INVALID from the host checks just past it."""
    import re
    import torch
    from paper_2203_03732_gb300 import _lib
    L = _lib.load()
    dummy = torch.zeros(64, dtype=torch.float64, device="cuda")
    st = _lib.PrStats()
    rc = L.pr_assign(dummy.data_ptr(), 1, 1 << 23, 4, 1 << 23, 0.1, dummy.data_ptr(), dummy.data_ptr(),
                     dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), ctypes.byref(st), None, 0, None)
    assert rc == _lib.PR_ERR_INVALID
    nmax = int(re.search(rb"max (\d+)", L.pr_last_error()).group(1))
    assert 50000 < nmax < (1 << 20)
    C = W.assignment_euclid_2d(40, 17, n_a=nmax)
    got = gpu_solve(prot, C, 0.1)
    assert_parity(got, oracle.assign(C, 0.1))
    C2 = torch.rand(2, nmax + 32, dtype=torch.float64, device="cuda")
    with pytest.raises(prot.PrError) as e:
        prot.assign(C2, 0.1)
    assert e.value.status == _lib.PR_ERR_INVALID


def test_pinned_host_costs_read_in_place(prot):
    """C in pinned host memory: the rounding kernel reads it over the host
    link, and the result equals the oracle's; pageable host memory is
    refused on the host (PR_ERR_INVALID), before any kernel runs."""
    import torch
    from paper_2203_03732_gb300 import _lib
    C = W.assignment_euclid_2d(1500, 23)
    Cp = torch.from_numpy(C).pin_memory()
    L = _lib.load()
    n = 1500
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4)]
    cst = torch.empty((), dtype=torch.float64, device="cuda")
    wsp = torch.empty(L.pr_assign_workspace(n, n), dtype=torch.uint8, device="cuda")
    st = _lib.PrStats()
    rc = L.pr_assign(Cp.data_ptr(), 1, n, n, n, 0.01, outs[0].data_ptr(), outs[1].data_ptr(),
                     outs[2].data_ptr(), outs[3].data_ptr(), cst.data_ptr(), ctypes.byref(st),
                     wsp.data_ptr(), wsp.numel(), None)
    assert rc == _lib.PR_OK
    ref = oracle.assign(C, 0.01)
    for k, t in zip(("row_to_col", "col_to_row", "y_row", "y_col"), outs):
        assert np.array_equal(t.cpu().numpy(), ref[k]), k
    assert st.phases == ref["stats"]["phases"]
    assert abs(float(cst) - ref["cost"]) <= COST_RTOL * ref["cost"]
    r2 = prot.assign(Cp, 0.01, results_on_device=True)
    assert r2["row_to_col"].is_cuda and np.array_equal(r2["row_to_col"].cpu().numpy(), ref["row_to_col"])
    # pageable host memory through the C ABI
    Ch = np.ascontiguousarray(C[:50, :50])
    out = [torch.empty(50, dtype=torch.int32, device="cuda") for _ in range(4)]
    cost = torch.empty((), dtype=torch.float64, device="cuda")
    ws = torch.empty(L.pr_assign_workspace(50, 50), dtype=torch.uint8, device="cuda")
    st = _lib.PrStats()
    rc = L.pr_assign(Ch.ctypes.data, 1, 50, 50, 50, 0.1, out[0].data_ptr(), out[1].data_ptr(),
                     out[2].data_ptr(), out[3].data_ptr(), cost.data_ptr(), ctypes.byref(st),
                     ws.data_ptr(), ws.numel(), None)
    assert rc == _lib.PR_ERR_INVALID
    assert b"pinned host memory" in L.pr_last_error()
    torch.cuda.synchronize()


@pytest.mark.parametrize("nB,nA,eps", [(3900, 3900, 0.003), (8000, 8000, 0.02), (6000, 9500, 0.01)])
def test_barrier_places_the_pool(prot, monkeypatch, nB, nA, eps):
    """Rows long enough that no CTA keeps rows for its next phase, so the grid
    barrier's arrival places each CTA's pool donations and a reader may find
    a slot still free and wait for it: 16-bit storage (eps = 0.003), bytes,
    and more columns than rows; bit-exact with the oracle, entries examined
    included."""
    set_form(monkeypatch, "grid")
    C = W.assignment_euclid_2d(nB, 7 + nB, n_a=nA)
    got = gpu_solve(prot, C, eps)
    assert_parity(got, oracle.assign(C, eps))
    assert_cells(got, C, eps)
