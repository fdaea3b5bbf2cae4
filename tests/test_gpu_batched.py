"""GPU parity of the batched solvers (pr_assign_batched, pr_assign_batched_points)
against the CPU oracle, problem by problem: bit-exact matching, duals and
phase count; FP64 cost within 1e-12 relative."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import points as OP
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


def check_problem(got, i, off, n, ref):
    sl = slice(off, off + n)
    for k in ("row_to_col", "col_to_row", "y_row", "y_col"):
        assert np.array_equal(got[k][sl], ref[k]), f"problem {i}: {k} differs"
    assert got["phases"][i] == ref["stats"]["phases"], f"problem {i}: phases"
    assert abs(got["costs"][i] - ref["cost"]) <= COST_RTOL * max(abs(ref["cost"]), 1e-300)


@pytest.mark.parametrize("threads", [128, 256, 1024])
def test_matrix_batch_matches_oracle(prot, threads):
    import torch
    sizes = np.array([1, 7, 64, 300, 513, 1000, 33, 2048], np.int32)
    eps = 0.01
    mats = [W.assignment_euclid_2d(int(n), 40 + i) for i, n in enumerate(sizes)]
    packed = np.concatenate([m.ravel() for m in mats])
    got = prot.assign_batched(torch.from_numpy(packed).cuda(), sizes, eps,
                              tune=(threads, 0))
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in got.items()}
    off = 0
    for i, n in enumerate(sizes):
        ref = oracle.assign(mats[i], eps)
        check_problem(got, i, off, int(n), ref)
        off += int(n)


@pytest.mark.parametrize("eps", [0.1, 0.01, 0.005, 0.003])
def test_points_batch_matches_oracle(prot, eps):
    """Byte storage with the plain-add pre-test (eps 0.1, 0.01), with the
    carry-isolated one (0.005), and 16-bit storage (0.003)."""
    import torch
    sizes = W.batched_sizes(24, 64, 700, seed=5)
    XA, XB, off = W.batched_points_3d(sizes, seed=5)
    got = prot.assign_batched_points(torch.from_numpy(XA).cuda(), torch.from_numpy(XB).cuda(),
                                     sizes, eps, metric="sqeuclidean")
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in got.items()}
    for i, n in enumerate(sizes):
        s, e = off[i], off[i + 1]
        ref = OP.assign_points(XA[s:e], XB[s:e], eps, squared=True)
        check_problem(got, i, int(s), int(n), ref)


@pytest.mark.parametrize("dim,metric", [(2, "euclidean"), (5, "sqeuclidean"), (1, "euclidean")])
def test_points_other_dimensions(prot, dim, metric):
    """Two dimensions (its own kernel), and five and one (the kernel for any
    dimension): the same costs, bit for bit, as the oracle's point solve."""
    import torch
    sizes = W.batched_sizes(12, 33, 400, seed=dim)
    g = np.random.default_rng(100 + dim)
    total = int(np.sum(sizes))
    XA = g.random((total, dim)).astype(np.float32)
    XB = g.random((total, dim)).astype(np.float32)
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    got = prot.assign_batched_points(torch.from_numpy(XA).cuda(), torch.from_numpy(XB).cuda(),
                                     sizes, 0.02, metric=metric)
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in got.items()}
    for i, n in enumerate(sizes):
        s, e = off[i], off[i + 1]
        ref = OP.assign_points(XA[s:e], XB[s:e], 0.02, squared=metric == "sqeuclidean")
        check_problem(got, i, int(s), int(n), ref)


def test_points_euclidean_and_float32_matrix(prot):
    import torch
    sizes = np.array([100, 257, 64], np.int32)
    XA, XB, off = W.batched_points_3d(sizes, seed=9)
    got = prot.assign_batched_points(torch.from_numpy(XA).cuda(), torch.from_numpy(XB).cuda(),
                                     sizes, 0.02, metric="euclidean")
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in got.items()}
    for i, n in enumerate(sizes):
        s, e = off[i], off[i + 1]
        ref = OP.assign_points(XA[s:e], XB[s:e], 0.02, squared=False)
        check_problem(got, i, int(s), int(n), ref)
    # the FP32 cost matrices of those problems through the matrix entry point
    mats = [OP.cost_matrix(XA[off[i]:off[i + 1]], XB[off[i]:off[i + 1]], squared=False)
            for i in range(len(sizes))]
    packed = np.concatenate([m.ravel() for m in mats])
    got2 = prot.assign_batched(torch.from_numpy(packed).cuda(), sizes, 0.02)
    for i, n in enumerate(sizes):
        ref = oracle.assign(mats[i], 0.02)
        s = int(off[i])
        assert np.array_equal(got2["row_to_col"].cpu().numpy()[s:s + n], ref["row_to_col"])
        assert np.array_equal(got2["y_row"].cpu().numpy()[s:s + n], ref["y_row"])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_matrix_batch_sixteen_bit_storage(prot, dtype):
    """eps = 0.003 (floor(1/eps) = 333 > 252): the matrix rounding writes
    16-bit values; FP64 and FP32 matrices, sizes with ragged rows."""
    import torch
    sizes = np.array([5, 63, 130, 301], np.int32)
    eps = 0.003
    mats = [W.assignment_euclid_2d(int(n), 70 + i).astype(dtype) for i, n in enumerate(sizes)]
    packed = np.concatenate([m.ravel() for m in mats])
    got = prot.assign_batched(torch.from_numpy(packed).cuda(), sizes, eps)
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in got.items()}
    off = 0
    for i, n in enumerate(sizes):
        check_problem(got, i, off, int(n), oracle.assign(mats[i], eps))
        off += int(n)


def test_matrix_batch_refuses_a_cost_out_of_range(prot):
    """One cost above 1 in one problem of the batch: PR_ERR_INVALID."""
    import torch
    sizes = np.array([40, 70, 33], np.int32)
    mats = [W.assignment_euclid_2d(int(n), 90 + i) for i, n in enumerate(sizes)]
    mats[1][17, 5] = 1.5
    packed = np.concatenate([m.ravel() for m in mats])
    with pytest.raises(prot.PrError) as e:
        prot.assign_batched(torch.from_numpy(packed).cuda(), sizes, 0.05)
    assert e.value.status == -1


def test_batch_equals_single_problem_solver(prot):
    """Closed form (v): each batched result equals pr_assign on that problem."""
    import torch
    sizes = np.array([800, 1500, 96], np.int32)
    mats = [W.assignment_euclid_2d(int(n), 70 + i) for i, n in enumerate(sizes)]
    packed = np.concatenate([m.ravel() for m in mats])
    got = prot.assign_batched(torch.from_numpy(packed).cuda(), sizes, 0.01)
    off = 0
    for i, n in enumerate(sizes):
        single = prot.assign(torch.from_numpy(mats[i]).cuda(), 0.01)
        for k in ("row_to_col", "col_to_row", "y_row", "y_col"):
            assert torch.equal(got[k][off:off + n], single[k])
        assert int(got["phases"][i]) == single["stats"]["phases"]
        off += int(n)


def test_config_sized_batch_sampled(prot):
    """The 512-problem point-cloud workload (n_i uniform in [64, 2048], 3-D,
    squared Euclidean, eps = 0.01) in the launch the bench times; a sample of
    problems is compared with the oracle."""
    import torch
    sizes = W.batched_sizes(512, 64, 2048, seed=0)
    XA, XB, off = W.batched_points_3d(sizes, seed=0)
    got = prot.assign_batched_points(torch.from_numpy(XA).cuda(), torch.from_numpy(XB).cuda(),
                                     sizes, 0.01, metric="sqeuclidean")
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in got.items()}
    rng = np.random.default_rng(1)
    sample = sorted(set(rng.choice(512, size=10, replace=False).tolist()) |
                    {int(np.argmax(sizes)), int(np.argmin(sizes))})
    for i in sample:
        s, e = off[i], off[i + 1]
        ref = OP.assign_points(XA[s:e], XB[s:e], 0.01, squared=True)
        check_problem(got, i, int(s), int(sizes[i]), ref)
    # every problem: a perfect matching
    for i in range(512):
        s, e = int(off[i]), int(off[i + 1])
        assert sorted(got["row_to_col"][s:e].tolist()) == list(range(e - s))


def test_batched_bad_sizes(prot):
    import torch
    with pytest.raises(prot.PrError):
        prot.assign_batched(torch.zeros(4, dtype=torch.float64, device="cuda"),
                            np.array([0, 2], np.int32), 0.1)
    with pytest.raises((prot.PrError, ValueError)):
        prot.assign_batched(torch.zeros(36000000, dtype=torch.float64, device="cuda"),
                            np.array([6000], np.int32), 0.1)


def test_autotune_picks_a_shape_and_keeps_results(prot, tmp_path, monkeypatch):
    """The library's autotuner times every launch shape on the batch; the
    chosen shape is cached, and the results equal the oracle's."""
    import json
    import torch
    monkeypatch.setenv("PROT_TUNE_CACHE", str(tmp_path / "tune.json"))
    sizes = W.batched_sizes(40, 64, 900, seed=12)
    XA, XB, off = W.batched_points_3d(sizes, seed=12)
    XAd, XBd = torch.from_numpy(XA).cuda(), torch.from_numpy(XB).cuda()
    got = prot.assign_batched_points(XAd, XBd, sizes, 0.01, tune="auto")
    cache = json.load(open(tmp_path / "tune.json"))
    assert len(cache) == 1
    threads, per_sm = next(iter(cache.values()))
    assert threads in (128, 256, 512, 1024) and 1 <= per_sm <= 4
    got = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in got.items()}
    for i in (0, 7, 39):
        s, e = off[i], off[i + 1]
        ref = OP.assign_points(XA[s:e], XB[s:e], 0.01, squared=True)
        check_problem(got, i, int(s), int(sizes[i]), ref)
    # a second call reads the cache and gives the same result
    again = prot.assign_batched_points(XAd, XBd, sizes, 0.01, tune="auto")
    assert np.array_equal(again["row_to_col"].cpu().numpy(), got["row_to_col"])
