"""GPU parity of pr_assign_points (costs formed on the device from point
sets) against the oracle's point-cloud solve: bit-exact matching, both dual
vectors, phases and rounds; FP64 cost within 1e-12 relative.  The costs
follow the oracle's points reading: FP32 distances one IEEE operation at a
time, c = RN32(d / max d), Eq. (1) on c."""
import numpy as np
import pytest

import oracle
from oracle import points as opoints
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


def check(prot, XA, XB, eps, metric):
    import torch
    got = prot.assign_points(torch.from_numpy(XA).cuda(), torch.from_numpy(XB).cuda(), eps, metric=metric)
    ref = opoints.assign_points(XA, XB, eps, squared=(metric == "sqeuclidean"))
    for k in ("row_to_col", "col_to_row", "y_row", "y_col"):
        assert np.array_equal(got[k].cpu().numpy(), ref[k]), k
    assert got["stats"]["phases"] == ref["stats"]["phases"]
    assert got["stats"]["rounds"] == ref["stats"]["rounds"]
    c = float(got["cost"].cpu())
    assert abs(c - ref["cost"]) <= 1e-12 * max(abs(ref["cost"]), 1e-300)
    return got


@pytest.mark.parametrize("n,dim,metric,eps", [
    (1000, 2, "euclidean", 0.1), (2049, 3, "sqeuclidean", 0.01), (5003, 2, "euclidean", 0.005),
    (700, 1, "euclidean", 0.02), (900, 17, "sqeuclidean", 0.05), (64, 2, "euclidean", 0.01)])
def test_parity(prot, n, dim, metric, eps):
    A, B = W.points_uniform(n, n, dim, 70 + n, dtype=np.float32)
    check(prot, A, B, eps, metric)


def test_unbalanced(prot):
    A, B = W.points_uniform(1500, 700, 3, 9, dtype=np.float32)
    check(prot, A, B, 0.02, "euclidean")


def test_full_size_n10000(prot):
    """The paper's synthetic workload (Sec. 5: uniform points in the unit
    square, Euclidean cost) at n = 10,000, eps = 0.01, costs from points."""
    A, B = W.points_uniform(10000, 10000, 2, 0, dtype=np.float32)
    check(prot, A, B, 0.01, "euclidean")


def test_same_solve_as_the_fp32_matrix(prot):
    """The points path and pr_assign on the oracle's FP32 cost matrix of the
    same points agree on the matching, both duals and the phase count."""
    import torch
    A, B = W.points_uniform(1200, 1200, 2, 3, dtype=np.float32)
    C = opoints.cost_matrix(A, B, squared=False)
    r1 = prot.assign_points(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 0.01)
    r2 = prot.assign(torch.from_numpy(C).cuda(), 0.01)
    for k in ("row_to_col", "col_to_row", "y_row", "y_col"):
        assert torch.equal(r1[k], r2[k]), k
    assert r1["stats"]["phases"] == r2["stats"]["phases"]
    assert r1["stats"]["cells_examined"] == r2["stats"]["cells_examined"]


def test_coincident_points(prot):
    """All distances 0 (max d = 0, every cost 0): one phase of n rounds that
    gives the identity, as for a zero cost matrix."""
    A = np.full((300, 2), 0.25, np.float32)
    B = A.copy()
    got = check(prot, A, B, 0.1, "euclidean")
    assert got["row_to_col"].cpu().tolist() == list(range(300))


def test_non_finite_coordinates_reported(prot):
    import torch
    A, B = W.points_uniform(200, 200, 2, 1, dtype=np.float32)
    B[17, 1] = np.nan
    with pytest.raises(prot.PrError) as e:
        prot.assign_points(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 0.1)
    assert e.value.status == -1
    A[3, 0] = np.inf
    B[17, 1] = 0.5
    with pytest.raises(prot.PrError):
        prot.assign_points(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 0.1)


def test_host_points_round_trip(prot):
    import torch
    A, B = W.points_uniform(800, 800, 2, 4, dtype=np.float32)
    got = prot.assign_points(torch.from_numpy(A), torch.from_numpy(B), 0.05)
    assert not got["row_to_col"].is_cuda
    ref = opoints.assign_points(A, B, 0.05, squared=False)
    assert np.array_equal(got["row_to_col"].numpy(), ref["row_to_col"])
