"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the method's arithmetic: it only draws points and
masses and, for the plain-solve workloads, forms the cost matrix the solver is
given as input (the paper's Sec. 5 synthetic experiment: points uniform in the
unit square, Euclidean cost).  Every generator uses numpy's PCG64 with an
explicit seed and draws the demand set A before the supply set B, so the same
bytes feed both sides.

Rows of every cost matrix are the supply vertices B (the side whose free
vertices propose), columns the demand vertices A: ``C[b, a] = c(a, b)``.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def points_uniform(n_a: int, n_b: int, dim: int, seed: int, dtype=np.float64):
    """A then B, i.i.d. uniform in [0, 1]^dim (Sec. 5, synthetic inputs)."""
    g = rng(seed)
    A = g.random((n_a, dim), dtype=np.float64)
    B = g.random((n_b, dim), dtype=np.float64)
    return A.astype(dtype), B.astype(dtype)


def points_normal(n_a: int, n_b: int, dim: int, seed: int, dtype=np.float32):
    g = rng(seed)
    A = g.standard_normal((n_a, dim), dtype=np.float64)
    B = g.standard_normal((n_b, dim), dtype=np.float64)
    return A.astype(dtype), B.astype(dtype)


def pairwise_cost(A: np.ndarray, B: np.ndarray, squared: bool, block: int = 1024) -> np.ndarray:
    """C[b, a] = |B[b] - A[a]|^2 (squared) or its IEEE sqrt, FP64, then
    divided by the matrix maximum so the largest cost is exactly 1 (Sec. 1).

    Coordinates are summed in ascending dimension order, one IEEE operation
    at a time (numpy evaluates each ufunc separately: no fused multiply-add).
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    nB, nA = B.shape[0], A.shape[0]
    C = np.empty((nB, nA), dtype=np.float64)
    for s in range(0, nB, block):
        e = min(nB, s + block)
        acc = None
        for d in range(A.shape[1]):
            diff = B[s:e, d][:, None] - A[:, d][None, :]
            sq = diff * diff
            acc = sq if acc is None else acc + sq
        C[s:e] = np.sqrt(acc) if not squared else acc
    m = C.max()
    if m > 0:
        for s in range(0, nB, block):
            C[s:s + block] /= m
    return C


def dirichlet1(n: int, g: np.random.Generator) -> np.ndarray:
    """Dirichlet(alpha = 1) masses as normalised Exp(1) draws, FP64."""
    x = g.standard_exponential(n)
    return x / x.sum()


# -------------------------------------------------------------------------
# The five synthetic workloads.
# -------------------------------------------------------------------------

def assignment_sq_euclid_2d(n: int, seed: int):
    """n points per side uniform in [0,1]^2, squared Euclidean cost / max."""
    A, B = points_uniform(n, n, 2, seed)
    return pairwise_cost(A, B, squared=True)


def assignment_euclid_2d(n: int, seed: int, n_a: int | None = None):
    """Points uniform in [0,1]^2, Euclidean cost / max (Sec. 5 synthetic)."""
    A, B = points_uniform(n if n_a is None else n_a, n, 2, seed)
    return pairwise_cost(A, B, squared=False)


def ot_euclid_2d(n_sup: int, n_dem: int, seed: int):
    """Points uniform in [0,1]^2, Euclidean cost / max, Dirichlet(1) supply
    and demand masses each summing to 1.  Returns (C, supply, demand)."""
    g = rng(seed)
    A = g.random((n_dem, 2))
    B = g.random((n_sup, 2))
    demand = dirichlet1(n_dem, g)
    supply = dirichlet1(n_sup, g)
    return pairwise_cost(A, B, squared=False), supply, demand


def batched_sizes(n_problems: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Problem sizes uniform integer in [lo, hi]."""
    return rng(seed).integers(lo, hi + 1, size=n_problems).astype(np.int32)


def batched_points_3d(sizes: np.ndarray, seed: int):
    """For each problem i: A_i, B_i with sizes[i] points uniform in [0,1]^3,
    FP32, packed back to back (A_0, A_1, ...; B_0, B_1, ...).
    Returns (XA, XB, off) with off[i] the first point of problem i."""
    g = rng(seed + 1)
    total = int(np.sum(sizes))
    XA = np.empty((total, 3), np.float32)
    XB = np.empty((total, 3), np.float32)
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    for i, n in enumerate(sizes):
        XA[off[i]:off[i + 1]] = g.random((n, 3), dtype=np.float64).astype(np.float32)
        XB[off[i]:off[i + 1]] = g.random((n, 3), dtype=np.float64).astype(np.float32)
    return XA, XB, off


def cloud_pairs_normal(batch: int, n: int, dim: int, seed: int):
    """batch pairs of point clouds, coordinates ~ N(0, 1), FP32: (X, Y)."""
    g = rng(seed)
    X = g.standard_normal((batch, n, dim), dtype=np.float64).astype(np.float32)
    Y = g.standard_normal((batch, n, dim), dtype=np.float64).astype(np.float32)
    return X, Y


# -------------------------------------------------------------------------
# MNIST-shaped synthetic images (the dataset itself is not available): the
# paper's second experiment matches n = 10,000 28x28 gray-level digit images
# of A against n of B, each normalised to unit mass, under the L1 distance
# (at most 2), for eps in {0.75, 0.5, 0.25, 0.1}.
# -------------------------------------------------------------------------

def mnist_shaped(n: int, seed: int, strokes=(1, 3), samples: int = 40, sigma: float = 0.9,
                 chunk: int = 256) -> np.ndarray:
    """n seeded 28x28 stroke images, flattened to (n, 784) FP64, each
    summing to 1.  An image is 1..3 quadratic Bezier strokes with control
    points in the central 20x20 box, drawn by a Gaussian brush of width
    sigma at `samples` points per stroke, clipped to [0, 1] gray levels with
    faint pixels set to 0 (about a fifth of the pixels are lit, as in
    handwritten digits)."""
    g = rng(seed)
    ns = g.integers(strokes[0], strokes[1] + 1, size=n)
    ctrl = g.uniform(4.0, 24.0, size=(n, strokes[1], 3, 2))
    t = np.linspace(0.0, 1.0, samples)[:, None]
    grid = np.arange(28.0)
    out = np.empty((n, 784))
    for i0 in range(0, n, chunk):
        c = ctrl[i0:i0 + chunk]                                       # (m, S, 3, 2)
        p0, p1, p2 = c[:, :, 0, None, :], c[:, :, 1, None, :], c[:, :, 2, None, :]
        pts = (1 - t) ** 2 * p0 + 2 * (1 - t) * t * p1 + t ** 2 * p2  # (m, S, samples, 2)
        lit = (np.arange(strokes[1])[None, :] < ns[i0:i0 + chunk, None]).astype(np.float64)
        # the brush is separable: exp(-(dy^2 + dx^2) / 2 s^2) = gy * gx
        gy = np.exp(-(pts[..., 0, None] - grid) ** 2 / (2 * sigma * sigma)) * lit[:, :, None, None]
        gx = np.exp(-(pts[..., 1, None] - grid) ** 2 / (2 * sigma * sigma))
        img = np.einsum("msti,mstj->mij", gy, gx).reshape(c.shape[0], 784)
        img = np.clip(img, 0.0, 1.0)
        img[img < 0.1] = 0.0
        out[i0:i0 + chunk] = img
    return out / out.sum(axis=1, keepdims=True)


def l1_cost(A: np.ndarray, B: np.ndarray, block: int = 32) -> np.ndarray:
    """C[b, a] = sum_k |B[b, k] - A[a, k]| in FP64 (numpy order), divided by
    the matrix maximum so that the largest cost is 1 (Sec. 1)."""
    C = np.empty((B.shape[0], A.shape[0]))
    for b0 in range(0, B.shape[0], block):
        C[b0:b0 + block] = np.abs(B[b0:b0 + block, None, :] - A[None, :, :]).sum(-1)
    m = C.max()
    return C / m if m > 0 else C


def mnist_shaped_pair(n: int, seed: int):
    """A then B, n images each: (A, B) as (n, 784) FP64 unit-mass rows."""
    return mnist_shaped(n, seed), mnist_shaped(n, seed + 7919)
