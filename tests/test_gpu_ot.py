"""GPU parity of pr_ot against the OT oracle: cluster duals, phase and round
counts bit-exact; the plan (masses after the fix-up) bit-exact; FP64 cost
within 1e-12 relative; plan feasibility."""
import numpy as np
import pytest

import oracle
from oracle import ot as O
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


def gpu_ot(P, C, nu, mu, eps):
    import torch
    r = P.ot(torch.from_numpy(C).cuda(), torch.from_numpy(nu).cuda(), torch.from_numpy(mu).cuda(), eps)
    nB, nA = C.shape
    dense = np.zeros((nB, nA))
    rows, cols = r["plan_row"].cpu().numpy(), r["plan_col"].cpu().numpy()
    assert len(set(zip(rows.tolist(), cols.tolist()))) == rows.size  # each pair once
    dense[rows, cols] = r["plan_mass"].cpu().numpy()
    return r, dense


def assert_ot_parity(r, dense, ref):
    assert np.array_equal(r["y_sup"].cpu().numpy(), ref["F"])
    assert np.array_equal(r["dem_kmin"].cpu().numpy(), ref["kmin"])
    assert np.array_equal(r["dem_lo"].cpu().numpy(), ref["clo"])
    assert np.array_equal(r["dem_hi"].cpu().numpy(), ref["chi"])
    st = r["stats"]
    assert st["phases"] == ref["stats"]["phases"]
    assert st["rounds"] == ref["stats"]["rounds"]
    assert st["free_at_stop"] == ref["stats"]["free_at_stop"]
    assert st["threshold"] == ref["T"]
    assert np.array_equal(dense, ref["mass"])
    c = float(r["cost"].cpu())
    assert abs(c - ref["cost"]) <= 1e-12 * abs(ref["cost"])
    assert_free_copies_feasible(r, ref["cbar"])


def assert_free_copies_feasible(r, cb, rows=512):
    """Eq. 2 between each supply's returned dual F_b (its free copies' dual)
    and the highest dual among each demand's copies: F_b + y(a) <= cbar + 1
    in units of eps, from the GPU's own outputs.  A demand of zero mass has
    no copies (D_a = ceil(theta * 0) = 0, Sec. 4), so no edge of the copy
    instance ends at it and it is left out."""
    F = r["y_sup"].cpu().numpy().astype(np.int64)
    kmin = r["dem_kmin"].cpu().numpy().astype(np.int64)
    lo = r["dem_lo"].cpu().numpy()
    has = (lo + r["dem_hi"].cpu().numpy()) > 0
    top = np.where(lo > 0, -kmin, -kmin - 1)
    for b0 in range(0, F.size, rows):
        blk = cb[b0:b0 + rows].astype(np.int64)
        assert not ((F[b0:b0 + rows, None] + top[None, :] > blk + 1) & has[None, :]).any()


@pytest.mark.parametrize("nB,nA,eps", [(20, 25, 0.1), (64, 64, 0.05), (300, 257, 0.05),
                                       (1000, 1200, 0.02), (2100, 2000, 0.1), (1, 1, 0.5)])
def test_ot_matches_oracle(prot, nB, nA, eps):
    C, nu, mu = W.ot_euclid_2d(nB, nA, nB + nA)
    r, dense = gpu_ot(prot, C, nu, mu, eps)
    ref = O.ot(C, nu, mu, eps)
    assert_ot_parity(r, dense, ref)
    assert np.abs(dense.sum(1) - nu).max() <= 1e-12
    assert (dense.sum(0) - mu).max() <= 1e-12


def test_ot_zero_masses(prot):
    C, nu, mu = W.ot_euclid_2d(40, 50, 3)
    nu = nu.copy()
    nu[[1, 7]] = 0.0
    nu /= nu.sum()
    mu = mu.copy()
    mu[[0, 4, 49]] = 0.0
    mu /= mu.sum()
    r, dense = gpu_ot(prot, C, nu, mu, 0.05)
    assert_ot_parity(r, dense, O.ot(C, nu, mu, 0.05))


def test_ot_full_size(prot):
    """The 10,000 x 10,000 Dirichlet(1) workload at eps = 0.05, compared in full."""
    C, nu, mu = W.ot_euclid_2d(10000, 10000, 0)
    r, dense = gpu_ot(prot, C, nu, mu, 0.05)
    ref = O.ot(C, nu, mu, 0.05)
    assert_ot_parity(r, dense, ref)


def test_ot_bad_masses(prot):
    import torch
    C, nu, mu = W.ot_euclid_2d(10, 10, 1)
    nu[3] = -0.1
    with pytest.raises(prot.PrError):
        prot.ot(torch.from_numpy(C).cuda(), torch.from_numpy(nu).cuda(), torch.from_numpy(mu).cuda(), 0.1)


def test_ot_refuses_mass_sums(prot):
    """A side whose masses sum to more than 1.5 (exactly: whose floor(m 2^32)
    sum to 1.5 * 2^32 or more), or a mass of 2 or more, is refused with
    PR_ERR_INVALID (what passes keeps the fix-up's 2^-62 units below 2^63);
    the oracle refuses the same inputs."""
    import torch
    C, nu, mu = W.ot_euclid_2d(10, 12, 1)
    for bad_nu, bad_mu in ((nu * 1.6, mu), (nu, mu * 1.6), (np.r_[2.0, nu[1:]], mu)):
        with pytest.raises(prot.PrError) as e:
            prot.ot(torch.from_numpy(C).cuda(), torch.from_numpy(bad_nu).cuda(),
                    torch.from_numpy(bad_mu).cuda(), 0.1)
        assert e.value.status == -1
        with pytest.raises(ValueError):
            O.counts(bad_nu, bad_mu, 0.1)
    # below 1.5 is accepted (more demand than supply: every supply copy can match)
    r, dense = gpu_ot(prot, C, nu, mu * 1.4, 0.1)
    assert_ot_parity(r, dense, O.ot(C, nu, mu * 1.4, 0.1))


@pytest.mark.parametrize("nB,nA,eps", [(64, 128, 0.25), (128, 64, 0.1), (128, 256, 0.3)])
def test_ot_uniform_masses(prot, nB, nA, eps):
    """Uniform masses 1/n: the residuals are whole multiples of one small
    unit, so supply and demand runs start at the same place in the
    north-west walk (3, 8 and 5 times in these cases: the demand start is
    then dropped), and many residuals are empty."""
    C = W.assignment_euclid_2d(nB, 17, n_a=nA)
    nu, mu = np.full(nB, 1.0 / nB), np.full(nA, 1.0 / nA)
    r, dense = gpu_ot(prot, C, nu, mu, eps)
    ref = O.ot(C, nu, mu, eps)
    assert_ot_parity(r, dense, ref)
    assert np.abs(dense.sum(1) - nu).max() <= 1e-12
    assert (dense.sum(0) - mu).max() <= 1e-12


@pytest.mark.parametrize("nB,nA,eps", [(1, 300, 0.1), (300, 1, 0.1), (2, 700, 0.05), (700, 3, 0.2)])
def test_ot_one_or_few_vertices_on_a_side(prot, nB, nA, eps):
    """Degenerate shapes: one supply vertex (its copies spread over every
    demand), one demand vertex (one winner per round), and two or three
    vertices on a side; the north-west prefix sums then have one to three
    entries on that side."""
    C, nu, mu = W.ot_euclid_2d(nB, nA, 21)
    r, dense = gpu_ot(prot, C, nu, mu, eps)
    assert_ot_parity(r, dense, O.ot(C, nu, mu, eps))
    assert np.abs(dense.sum(1) - nu).max() <= 1e-12
    assert (dense.sum(0) - mu).max() <= 1e-12


def test_ot_barrier_timeout_reported_not_hung(prot, monkeypatch):
    """The loop kernel's grid barriers wait at most PR_SPIN_LIMIT_CYCLES: with
    one cycle every CTA gives up at its first barrier, pr_ot returns
    PR_ERR_TIMEOUT and the next solve is exact."""
    import torch
    C, nu, mu = W.ot_euclid_2d(300, 257, 9)
    monkeypatch.setenv("PR_SPIN_LIMIT_CYCLES", "1")
    with pytest.raises(prot.PrError) as e:
        prot.ot(torch.from_numpy(C).cuda(), torch.from_numpy(nu).cuda(), torch.from_numpy(mu).cuda(), 0.05)
    assert e.value.status == -3
    monkeypatch.delenv("PR_SPIN_LIMIT_CYCLES")
    r, dense = gpu_ot(prot, C, nu, mu, 0.05)
    assert_ot_parity(r, dense, O.ot(C, nu, mu, 0.05))


@pytest.mark.parametrize("nB,nA,eps,seed", [(400, 300, 0.01, 5), (150, 600, 0.02, 6)])
def test_ot_many_phases(prot, nB, nA, eps, seed):
    """Small eps: many phases, cluster shifts and evictions in the loop kernel."""
    C, nu, mu = W.ot_euclid_2d(nB, nA, seed)
    r, dense = gpu_ot(prot, C, nu, mu, eps)
    ref = O.ot(C, nu, mu, eps)
    assert ref["stats"]["phases"] > 3
    assert_ot_parity(r, dense, ref)


@pytest.mark.parametrize("nB,nA", [(60, 50), (120, 90)])
def test_ot_sixteen_bit_storage(prot, nB, nA):
    """eps = 0.003 (floor(1/eps) = 333 > 252): rounded costs and keys stored in
    16 bits instead of bytes; thousands of phases."""
    C, nu, mu = W.ot_euclid_2d(nB, nA, 13)
    r, dense = gpu_ot(prot, C, nu, mu, 0.003)
    assert_ot_parity(r, dense, O.ot(C, nu, mu, 0.003))


def test_ot_async_enqueue(prot):
    """sync=False: pr_ot only enqueues (no stats); after the stream is done
    the plan, cost and duals equal the oracle's, and pr_ws_status reports no
    device error."""
    import torch
    C, nu, mu = W.ot_euclid_2d(300, 257, 31)
    ws = prot.Workspace()
    r = prot.ot(torch.from_numpy(C).cuda(), torch.from_numpy(nu).cuda(), torch.from_numpy(mu).cuda(), 0.05,
                ws=ws, sync=False)
    assert "stats" not in r
    prot.ws_status(ws)
    nnz = int(r["plan_nnz"].item())
    ref = O.ot(C, nu, mu, 0.05)
    dense = np.zeros(C.shape)
    dense[r["plan_row"][:nnz].cpu().numpy(), r["plan_col"][:nnz].cpu().numpy()] = r["plan_mass"][:nnz].cpu().numpy()
    assert np.array_equal(dense, ref["mass"])
    assert np.array_equal(r["y_sup"].cpu().numpy(), ref["F"])
    assert np.array_equal(r["dem_kmin"].cpu().numpy(), ref["kmin"])
    assert abs(float(r["cost"].cpu()) - ref["cost"]) <= 1e-12 * abs(ref["cost"])


@pytest.mark.parametrize("sync", [True, False])
def test_ot_plan_capacity_found_on_the_device(prot, sync):
    """A plan_cap below the plan's size: PR_ERR_CAPACITY (at once with stats,
    from pr_ws_status without), plan_nnz then holds more than plan_cap, and
    the next solve on the same workspace is exact."""
    import torch
    C, nu, mu = W.ot_euclid_2d(120, 90, 32)
    ref = O.ot(C, nu, mu, 0.05)
    need = int((ref["mass"] != 0).sum())
    args = (torch.from_numpy(C).cuda(), torch.from_numpy(nu).cuda(), torch.from_numpy(mu).cuda(), 0.05)
    ws = prot.Workspace()
    for cap in (need // 2, need - 1):
        with pytest.raises(prot.PrError) as e:
            r = prot.ot(*args, plan_cap=cap, ws=ws, sync=sync)
            if not sync:
                prot.ws_status(ws)
        assert e.value.status == -6
        if not sync:
            assert int(r["plan_nnz"].item()) > cap
    r, dense = gpu_ot(prot, C, nu, mu, 0.05)
    assert_ot_parity(r, dense, ref)
    r = prot.ot(*args, plan_cap=need, ws=ws)
    assert int(r["plan_nnz"].item()) == need
