"""GPU parity of the other rules of step (I) against the oracle: the
seeded-start-column rule (pr_assign_rule with PR_RULE_OFFSET, the oracle's
OR_MODE_OFFSET) in every phase-loop form, and Israeli and Itai's randomized
maximal matching (PR_RULE_ISRAELI_ITAI, OR_MODE_ISRAELI_ITAI): bit-exact
matching, both dual vectors, phase and round counts, and the exact number of
cost entries the scans pass."""
import numpy as np
import pytest

import oracle
from paper_2203_03732_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FORMS = ["grid", "grid-slots", "cluster"]


@pytest.fixture(scope="module")
def prot():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_03732_gb300 import build
    build.build()
    import paper_2203_03732_gb300 as P
    return P


def set_form(monkeypatch, form):
    monkeypatch.setenv("PR_PHASE_MODE", "cluster" if form == "cluster" else "grid")
    monkeypatch.setenv("PR_SCAN", "auto" if form == "grid-slots" else "regs")


MODES = {"offset": oracle.MODE_OFFSET, "israeli-itai": oracle.MODE_ISRAELI_ITAI,
         "sequential": oracle.MODE_SEQUENTIAL}


def check(prot, C, eps, rule="offset"):
    import torch
    r = prot.assign(torch.from_numpy(C).cuda(), eps, rule=rule)
    ref = oracle.assign(C, eps, mode=MODES[rule])
    for k in ("row_to_col", "col_to_row", "y_row", "y_col"):
        assert np.array_equal(r[k].cpu().numpy(), ref[k]), k
    for k in ("phases", "rounds", "free_at_stop"):
        assert r["stats"][k] == ref["stats"][k], k
    if rule == "sequential":
        # the chains resume where they lost a column; the oracle's greedy
        # rescans every row from column 0, so only the bound is shared
        assert 0 < r["stats"]["cells_examined"] <= ref["stats"]["scanned"]
    else:
        assert r["stats"]["cells_examined"] == ref["stats"]["scanned"]
    assert abs(float(r["cost"]) - ref["cost"]) <= 1e-12 * max(abs(ref["cost"]), 1e-300)
    return r, ref


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,eps", [(64, 0.1), (1000, 0.01), (4097, 0.005), (5003, 0.1), (700, 0.002)])
def test_offset_rule_parity(prot, monkeypatch, form, n, eps):
    set_form(monkeypatch, form)
    check(prot, W.assignment_euclid_2d(n, 90 + n), eps)


def test_offset_rule_unbalanced(prot):
    C = W.assignment_euclid_2d(900, 4, n_a=2300)
    for eps in (0.1, 0.02):
        check(prot, C, eps)


def test_offset_rule_full_size(prot):
    """n = 10,000 at eps = 0.1 (the paper's largest eps) with the offset rule."""
    r, _ = check(prot, W.assignment_euclid_2d(10000, 0), 0.1)
    low = oracle.assign(W.assignment_euclid_2d(10000, 0), 0.1)["stats"]
    assert r["stats"]["rounds"] * 3 < low["rounds"]


@pytest.mark.parametrize("eps", [0.75, 0.25])
def test_offset_rule_mnist_shaped(prot, eps):
    """Where most edges are admissible the rule needs far fewer rounds than
    the lowest-index rule, with the same guarantees (Lemma 3.1 bound)."""
    import torch
    A, B = W.mnist_shaped_pair(600, 5)
    C = W.l1_cost(A, B)
    r, _ = check(prot, C, eps)
    low = prot.assign(torch.from_numpy(C).cuda(), eps)
    if eps == 0.75:
        assert r["stats"]["rounds"] * 4 < low["stats"]["rounds"]
    opt, _ = oracle.hungarian(C)
    assert opt - 1e-9 <= float(r["cost"]) <= opt + 3 * eps * 600 + 1e-9


def test_bad_rule(prot):
    import ctypes
    import torch
    from paper_2203_03732_gb300 import _lib
    L = _lib.load()
    C = torch.rand(10, 10, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        prot.assign(C, 0.1, rule="random")
    st = _lib.PrStats()
    rc = L.pr_assign_rule(7, C.data_ptr(), 1, 10, 10, 10, 0.1, None, None, None, None, None,
                          ctypes.byref(st), None, 0, None)
    assert rc == _lib.PR_ERR_INVALID


# ---------------------------------------------------------------------------
# Israeli-Itai rounds (Sec. 3.2, parallel efficiency)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,eps", [(7, 0.1), (64, 0.1), (300, 0.02), (1000, 0.01), (2049, 0.005),
                                   (700, 0.002), (1500, 0.1)])
def test_israeli_itai_parity(prot, n, eps):
    """Byte and 16-bit storage (eps = 0.002), one and many phases, ragged
    row lengths: the GPU's rounds pick the oracle's edges."""
    check(prot, W.assignment_euclid_2d(n, 70 + n), eps, rule="israeli-itai")


def test_israeli_itai_unbalanced_and_fp32(prot):
    C = W.assignment_euclid_2d(400, 6, n_a=1100)
    check(prot, C, 0.05, rule="israeli-itai")
    check(prot, C.astype(np.float32), 0.02, rule="israeli-itai")


@pytest.mark.parametrize("eps", [0.75, 0.5, 0.1])
def test_israeli_itai_mnist_shaped(prot, eps):
    """Where most edges are admissible a phase takes a few rounds, against
    hundreds for the lowest-index rule; the Lemma 3.1 bound holds."""
    import torch
    A, B = W.mnist_shaped_pair(600, 5)
    C = W.l1_cost(A, B)
    r, _ = check(prot, C, eps, rule="israeli-itai")
    if eps == 0.75:
        low = prot.assign(torch.from_numpy(C).cuda(), eps)
        assert r["stats"]["rounds"] * 10 < low["stats"]["rounds"]
        assert r["stats"]["rounds"] <= 4 * np.log2(600)
    opt, _ = oracle.hungarian(C)
    assert opt - 1e-9 <= float(r["cost"]) <= opt + 3 * eps * 600 + 1e-9


def test_israeli_itai_repeatable(prot):
    """The draws are keyed, not taken from a device generator: two solves
    give the same bits."""
    import torch
    C = torch.from_numpy(W.assignment_euclid_2d(1200, 8)).cuda()
    a = prot.assign(C, 0.01, rule="israeli-itai")
    b = prot.assign(C, 0.01, rule="israeli-itai")
    for k in ("row_to_col", "y_row", "y_col"):
        assert torch.equal(a[k], b[k])


# ---------------------------------------------------------------------------
# The sequential greedy by displacement chains (Sec. 3.2), no rounds
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,eps", [(7, 0.1), (64, 0.1), (300, 0.02), (1000, 0.01), (2049, 0.005),
                                   (700, 0.002), (1500, 0.1), (5003, 0.01)])
def test_sequential_parity(prot, n, eps):
    """Byte and 16-bit storage (eps = 0.002), one and many phases, ragged
    row lengths: the chains end every phase with the oracle's greedy M'."""
    check(prot, W.assignment_euclid_2d(n, 50 + n), eps, rule="sequential")


def test_sequential_unbalanced_fp32_and_few_costs(prot):
    C = W.assignment_euclid_2d(400, 6, n_a=1100)
    check(prot, C, 0.05, rule="sequential")
    check(prot, C.astype(np.float32), 0.02, rule="sequential")
    g = np.random.default_rng(12)
    check(prot, g.integers(0, 4, size=(900, 900)) / 3.0, 0.1, rule="sequential")


@pytest.mark.parametrize("eps", [0.75, 0.25])
def test_sequential_mnist_shaped(prot, eps):
    """Where most edges are admissible many rows meet at the same columns,
    so the chains displace each other most; the result is still the
    greedy's, and the Lemma 3.1 bound holds."""
    import torch
    A, B = W.mnist_shaped_pair(600, 5)
    C = W.l1_cost(A, B)
    r, _ = check(prot, C, eps, rule="sequential")
    assert r["stats"]["rounds"] == r["stats"]["phases"]
    opt, _ = oracle.hungarian(C)
    assert opt - 1e-9 <= float(r["cost"]) <= opt + 3 * eps * 600 + 1e-9


def test_sequential_full_size(prot):
    """n = 10,000 at eps = 0.01 against the oracle's greedy."""
    check(prot, W.assignment_euclid_2d(10000, 0), 0.01, rule="sequential")


def test_sequential_repeatable(prot):
    """The scans race for columns, but the result does not depend on who
    wins when: ten solves give the same bits."""
    import torch
    C = torch.from_numpy(W.assignment_euclid_2d(3000, 9)).cuda()
    a = prot.assign(C, 0.01, rule="sequential")
    for _ in range(9):
        b = prot.assign(C, 0.01, rule="sequential")
        for k in ("row_to_col", "y_row", "y_col"):
            assert torch.equal(a[k], b[k])


def test_sequential_too_many_columns_refused(prot):
    """The phase's keys live in shared memory: more columns than fit are
    refused on the host, before anything runs."""
    import torch
    C = torch.zeros(1, 196624, dtype=torch.float32, device="cuda")
    with pytest.raises(prot.PrError) as e:
        prot.assign(C, 0.1, rule="sequential")
    assert e.value.status == -1
