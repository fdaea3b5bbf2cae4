"""CPU checks of the seeded synthetic generators that stand in for the
paper's inputs (no method arithmetic here)."""
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
