"""CPU checks of the seeded synthetic generators that stand in for the
paper's inputs (no method arithmetic here)."""
import math

import numpy as np

from paper_2203_03732_gb300 import workloads as W


def test_mnist_shaped_images():
    """28x28 non-negative images of unit mass, reproducible from the seed,
    about a fifth of the pixels lit (handwritten digits light ~19 %)."""
    A = W.mnist_shaped(300, 5)
    assert A.shape == (300, 784) and A.dtype == np.float64
    assert (A >= 0).all()
    assert np.allclose(A.sum(1), 1.0, rtol=0, atol=1e-12)
    lit = (A > 0).mean()
    assert 0.08 < lit < 0.35
    assert (A > 0).sum(1).min() >= 10
    assert np.array_equal(A, W.mnist_shaped(300, 5))
    assert not np.array_equal(A, W.mnist_shaped(300, 6))


def test_l1_cost_definition():
    """C[b, a] = sum_k |B[b] - A[a]| / max: brute force on a few rows, the
    largest entry exactly 1, and symmetric for A = B with a zero diagonal."""
    A, B = W.mnist_shaped_pair(40, 2)
    C = W.l1_cost(A, B)
    raw = np.array([[np.abs(B[b] - A[a]).sum() for a in range(40)] for b in range(40)])
    assert np.allclose(C, raw / raw.max(), rtol=1e-15, atol=0)
    assert C.max() == 1.0 and C.min() >= 0.0
    S = W.l1_cost(A, A)
    assert np.allclose(S, S.T) and np.all(np.diag(S) == 0.0)
    assert raw.max() <= 2.0 + 1e-12   # unit-mass images: L1 distance at most 2


def test_uniform_points_seeded_and_drawn_a_then_b():
    """Same seed, same bytes; A is drawn before B from one PCG64 stream;
    coordinates lie in [0, 1)."""
    A, B = W.points_uniform(5, 7, 2, 11)
    A2, B2 = W.points_uniform(5, 7, 2, 11)
    assert np.array_equal(A, A2) and np.array_equal(B, B2)
    g = np.random.Generator(np.random.PCG64(11))
    assert np.array_equal(A, g.random((5, 2))) and np.array_equal(B, g.random((7, 2)))
    assert A.min() >= 0.0 and B.max() < 1.0
    Af, _ = W.points_uniform(5, 7, 2, 11, dtype=np.float32)
    assert Af.dtype == np.float32 and np.array_equal(Af, A.astype(np.float32))


def test_pairwise_cost_rows_are_b_and_max_is_one():
    """C[b, a] is the distance from B[b] to A[a] (squared, or its square
    root) over the matrix maximum, so the largest cost is exactly 1 and every
    cost lies in [0, 1]; the coordinates are summed in ascending order."""
    A, B = W.points_uniform(4, 6, 3, 2)
    for squared in (True, False):
        C = W.pairwise_cost(A, B, squared=squared)
        assert C.shape == (6, 4) and C.max() == 1.0 and C.min() >= 0.0
        raw = np.empty((6, 4))
        for b in range(6):
            for a in range(4):
                s = 0.0
                for d in range(3):
                    t = B[b, d] - A[a, d]
                    s = s + t * t
                raw[b, a] = s if squared else math.sqrt(s)
        assert np.array_equal(C, raw / raw.max())


def test_ot_masses_and_costs():
    """Dirichlet(1) masses: positive, summing to 1 within rounding; costs in
    [0, 1] with maximum 1; shapes follow (n_sup, n_dem)."""
    C, nu, mu = W.ot_euclid_2d(9, 13, 4)
    assert C.shape == (9, 13) and C.max() == 1.0 and C.min() >= 0.0
    assert nu.shape == (9,) and mu.shape == (13,)
    assert (nu > 0).all() and (mu > 0).all()
    assert abs(nu.sum() - 1.0) < 1e-15 and abs(mu.sum() - 1.0) < 1e-15


def test_batched_and_cloud_generators():
    """Batched sizes lie in [lo, hi] and are seeded; the packed point sets
    follow the sizes; the autograd clouds are FP32 N(0, 1) draws."""
    s = W.batched_sizes(200, 64, 2048, 3)
    assert s.dtype == np.int32 and s.min() >= 64 and s.max() <= 2048
    assert np.array_equal(s, W.batched_sizes(200, 64, 2048, 3))
    sizes = np.array([3, 1, 4], np.int32)
    XA, XB, off = W.batched_points_3d(sizes, 0)
    assert off.tolist() == [0, 3, 4, 8] and XA.shape == XB.shape == (8, 3)
    assert XA.dtype == np.float32 and 0.0 <= XA.min() and XB.max() < 1.0
    X, Y = W.cloud_pairs_normal(2, 5, 3, 1)
    assert X.shape == Y.shape == (2, 5, 3) and X.dtype == np.float32
    g = np.random.Generator(np.random.PCG64(1))
    assert np.array_equal(X, g.standard_normal((2, 5, 3)).astype(np.float32))
