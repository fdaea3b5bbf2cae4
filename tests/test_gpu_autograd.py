"""GPU tests of the differentiable assignment loss: the forward plan and loss
match the oracle pair by pair, the hand-written backward kernel matches the
oracle gradient bit for bit, and on tiny inputs with a unique optimum the
gradient at the optimal plan equals finite differences of the exact loss."""
import itertools

import numpy as np
import pytest

from oracle import points as OP
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


def test_forward_and_backward_match_oracle(prot):
    import torch
    B, n, d, eps = 6, 300, 3, 0.01
    X, Y = W.cloud_pairs_normal(B, n, d, seed=3)
    Xt = torch.from_numpy(X).cuda().requires_grad_(True)
    Yt = torch.from_numpy(Y).cuda().requires_grad_(True)
    loss = prot.assignment_loss(Xt, Yt, eps)
    g = torch.linspace(0.5, 2.0, B, device="cuda")
    (loss * g).sum().backward()
    for p in range(B):
        ref = OP.assign_points(Y[p], X[p], eps, squared=True)  # columns = Y, rows = X
        assert abs(float(loss[p]) - np.float32(ref["cost"] / n)) <= 1e-6 * abs(ref["cost"] / n)
        gX, gY = OP.sqeuclid_backward(X[p], Y[p], ref["row_to_col"], float(g[p]))
        assert np.array_equal(Xt.grad[p].cpu().numpy(), gX)
        assert np.array_equal(Yt.grad[p].cpu().numpy(), gY)


def test_grad_c_and_permutation_property(prot):
    import torch
    B, n, d = 3, 64, 3
    X, Y = W.cloud_pairs_normal(B, n, d, seed=7)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    res = prot.assign_batched_points(Yt.reshape(-1, d), Xt.reshape(-1, d), [n] * B, 0.05)
    g = torch.tensor([1.0, -2.0, 0.25], device="cuda")
    gX, gY, gC = prot.assign_backward(res["row_to_col"], Xt, Yt, g, grad_C=True)
    r2c = res["row_to_col"].reshape(B, n)
    for p in range(B):
        # grad_Y[sigma(i)] == -grad_X[i]; grad_C is g/n on the plan, 0 elsewhere
        assert torch.equal(gY[p][r2c[p].long()], -gX[p])
        want = torch.zeros(n, n, device="cuda")
        want[torch.arange(n, device="cuda"), r2c[p].long()] = float(np.float32(float(g[p]) / n))
        assert torch.equal(gC[p], want)


def exact_plan(X, Y):
    n = X.shape[0]
    vals = []
    for perm in itertools.permutations(range(n)):
        vals.append((sum(float(np.sum((X[i].astype(np.float64) - Y[perm[i]]) ** 2)) for i in range(n)), perm))
    vals.sort()
    return np.array(vals[0][1], np.int32), (vals[1][0] - vals[0][0]) / n


def test_backward_kernel_at_exact_optimum_matches_finite_differences(prot):
    import torch
    g = np.random.default_rng(11)
    n, d = 5, 3
    for _ in range(50):
        X = g.standard_normal((1, n, d)).astype(np.float32)
        Y = g.standard_normal((1, n, d)).astype(np.float32)
        sigma, gap = exact_plan(X[0], Y[0])
        if gap > 1e-3:
            break
    gX, gY = prot.assign_backward(torch.from_numpy(sigma).cuda(), torch.from_numpy(X).cuda(),
                                  torch.from_numpy(Y).cuda(), torch.ones(1, device="cuda"))
    h = 1e-6
    X64, Y64 = X[0].astype(np.float64), Y[0].astype(np.float64)

    def loss(A, B_):
        return min(sum(float(np.sum((A[i] - B_[p[i]]) ** 2)) for i in range(n))
                   for p in itertools.permutations(range(n))) / n

    for i in range(n):
        for k in range(d):
            Xp, Xm = X64.copy(), X64.copy()
            Xp[i, k] += h
            Xm[i, k] -= h
            fd = (loss(Xp, Y64) - loss(Xm, Y64)) / (2 * h)
            assert abs(fd - float(gX[0, i, k])) < 1e-4 * max(1.0, abs(fd))


def test_config_sized_loss_sampled(prot):
    """The bench's differentiable-loss workload (64 pairs, n = 4096, d = 3,
    N(0,1) coordinates, squared Euclidean, eps = 0.01) in one batched
    forward + backward: four sampled pairs match the oracle's plan, loss and
    gradients bit for bit, and every pair's gradients obey grad_Y[sigma(i)] =
    -grad_X[i]."""
    import torch
    B, n, d, eps = 64, 4096, 3, 0.01
    X, Y = W.cloud_pairs_normal(B, n, d, seed=0)
    Xt = torch.from_numpy(X).cuda().requires_grad_(True)
    Yt = torch.from_numpy(Y).cuda().requires_grad_(True)
    loss = prot.assignment_loss(Xt, Yt, eps)
    loss.sum().backward()
    rng = np.random.default_rng(1)
    for p in sorted(rng.choice(B, size=4, replace=False).tolist()):
        ref = OP.assign_points(Y[p], X[p], eps, squared=True)
        assert abs(float(loss[p].detach()) - np.float32(ref["cost"] / n)) <= 1e-6 * abs(ref["cost"] / n)
        gX, gY = OP.sqeuclid_backward(X[p], Y[p], ref["row_to_col"], 1.0)
        assert np.array_equal(Xt.grad[p].cpu().numpy(), gX)
        assert np.array_equal(Yt.grad[p].cpu().numpy(), gY)
    res = prot.assign_batched_points(Yt.detach().reshape(-1, d), Xt.detach().reshape(-1, d), [n] * B, eps)
    r2c = res["row_to_col"].reshape(B, n).long()
    for p in range(B):
        assert torch.equal(Yt.grad[p][r2c[p]], -Xt.grad[p])
