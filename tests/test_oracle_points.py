"""Pins for the point-cloud oracle (CPU only): costs from points against an
independent numpy evaluation, and the gradient formula of the assignment loss
against central finite differences of the exact optimum (brute force)."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import points as OP
from paper_2203_03732_gb300 import workloads as W


def numpy_cost_f32(XA, XB, squared):
    XA = XA.astype(np.float32)
    XB = XB.astype(np.float32)
    acc = None
    for k in range(XA.shape[1]):
        t = (XB[:, k][:, None] - XA[:, k][None, :]).astype(np.float32)
        sq = (t * t).astype(np.float32)
        acc = sq if acc is None else (acc + sq).astype(np.float32)
    d = acc if squared else np.sqrt(acc).astype(np.float32)
    m = d.max()
    return (d / m).astype(np.float32) if m > 0 else np.zeros_like(d)


@pytest.mark.parametrize("squared", [True, False])
def test_points_cost_matches_numpy(squared):
    XA, XB = W.points_uniform(40, 33, 3, 2, dtype=np.float32)
    C = OP.cost_matrix(XA, XB, squared=squared)
    assert C.max() == np.float32(1.0)
    assert np.array_equal(C, numpy_cost_f32(XA, XB, squared))


def test_match_cost_fp64():
    XA, XB = W.points_uniform(20, 20, 3, 4, dtype=np.float32)
    perm = np.random.default_rng(0).permutation(20).astype(np.int32)
    want = sum(float(np.sum((XB[i].astype(np.float64) - XA[perm[i]].astype(np.float64)) ** 2))
               for i in range(20))
    assert abs(OP.match_cost(XA, XB, perm, squared=True) - want) <= 1e-14 * want


def test_points_solve_equals_matrix_solve():
    XA, XB = W.points_uniform(90, 90, 3, 6, dtype=np.float32)
    r = OP.assign_points(XA, XB, 0.02, squared=True)
    C = OP.cost_matrix(XA, XB, squared=True)
    m = oracle.assign(C, 0.02)
    assert np.array_equal(r["row_to_col"], m["row_to_col"])
    assert np.array_equal(r["y_row"], m["y_row"])
    assert r["stats"]["phases"] == m["stats"]["phases"]


def exact_loss(X, Y):
    """(1/n) min over permutations of sum |x_i - y_sigma(i)|^2 in FP64."""
    n = X.shape[0]
    best, arg = np.inf, None
    for perm in itertools.permutations(range(n)):
        v = sum(float(np.sum((X[i] - Y[perm[i]]) ** 2)) for i in range(n))
        if v < best:
            best, arg = v, perm
    return best / n, np.array(arg, np.int32)


def second_gap(X, Y):
    n = X.shape[0]
    vals = sorted(sum(float(np.sum((X[i] - Y[p[i]]) ** 2)) for i in range(n))
                  for p in itertools.permutations(range(n)))
    return (vals[1] - vals[0]) / n


@pytest.mark.parametrize("seed", range(4))
def test_gradient_formula_matches_finite_differences(seed):
    """At an input with a unique optimal plan (second-best gap > 1e-3), the
    closed-form gradient 2 (x_i - y_sigma(i)) / n equals the central finite
    difference (h = 1e-6) of the exact FP64 optimum."""
    g = np.random.default_rng(1000 + seed)
    n, d = 5, 3
    for _ in range(50):
        X = g.standard_normal((n, d))
        Y = g.standard_normal((n, d))
        if second_gap(X, Y) > 1e-3:
            break
    else:
        pytest.skip("no input with a unique optimum found")
    _, sigma = exact_loss(X, Y)
    gX, gY = OP.sqeuclid_backward(X.astype(np.float32), Y.astype(np.float32), sigma, 1.0)
    h = 1e-6
    for i in range(n):
        for k in range(d):
            for M, G in ((X, gX), (Y, gY)):
                row = i if M is X else int(sigma[i])
                Mp, Mm = M.copy(), M.copy()
                Mp[row, k] += h
                Mm[row, k] -= h
                fp = exact_loss(Mp, Y)[0] if M is X else exact_loss(X, Mp)[0]
                fm = exact_loss(Mm, Y)[0] if M is X else exact_loss(X, Mm)[0]
                fd = (fp - fm) / (2 * h)
                assert abs(fd - float(G[row, k])) < 1e-5 * max(1.0, abs(fd))


def test_backward_scales_with_upstream_gradient():
    X, Y = W.cloud_pairs_normal(1, 6, 3, 8)
    sigma = np.arange(6, dtype=np.int32)
    g1 = OP.sqeuclid_backward(X[0], Y[0], sigma, 1.0)
    g3 = OP.sqeuclid_backward(X[0], Y[0], sigma, -3.0)
    assert np.allclose(g3[0], -3.0 * g1[0], rtol=1e-6)
    # grad_Y[sigma(i)] == -grad_X[i]
    assert np.array_equal(g1[1][sigma], -g1[0])
