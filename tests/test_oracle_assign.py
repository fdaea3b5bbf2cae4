"""Pins for the assignment oracle (CPU only).

Every check here ties the oracle to something other than itself: brute force
over permutations, scipy's exact assignment solver, the paper's invariants
(I1)/(I2) and Lemma 2.1 after every phase, the bounds of Lemma 3.1, 3.2 and
Eq. (4), a hand-worked run of Sec. 2.2 (tests/golden), and closed forms.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2203_03732_gb300 import workloads as W

EPS_SET = [0.5, 0.3, 0.1, 0.05]


def brute_force(C):
    nB, nA = C.shape
    best = math.inf
    for perm in itertools.permutations(range(nA), nB):
        s = math.fsum(C[b, perm[b]] for b in range(nB))
        best = min(best, s)
    return best


def rand_costs(seed, nB, nA, kind="uniform"):
    g = np.random.default_rng(seed)
    if kind == "uniform":
        C = g.random((nB, nA))
    elif kind == "few":
        C = g.integers(0, 4, size=(nB, nA)) / 3.0
    else:
        raise ValueError(kind)
    return C


# -------------------------------------------------------------------------
# Exact solvers used as pins
# -------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_hungarian_matches_brute_force(seed):
    g = np.random.default_rng(seed)
    nB = int(g.integers(1, 7))
    nA = int(g.integers(nB, 8))
    C = rand_costs(seed, nB, nA, "uniform" if seed % 2 else "few")
    v, r2c = oracle.hungarian(C)
    assert len(set(r2c.tolist())) == nB
    assert abs(v - math.fsum(C[np.arange(nB), r2c])) < 1e-12
    assert abs(v - brute_force(C)) < 1e-12


@pytest.mark.parametrize("shape", [(40, 40), (120, 120), (60, 97), (300, 300)])
def test_hungarian_matches_scipy(shape):
    from scipy.optimize import linear_sum_assignment
    C = rand_costs(sum(shape), *shape)
    v, _ = oracle.hungarian(C)
    r, c = linear_sum_assignment(C)
    assert abs(v - C[r, c].sum()) < 1e-9


# -------------------------------------------------------------------------
# Eq. (1)
# -------------------------------------------------------------------------

def test_quantise_hand_values():
    C = np.array([[0.0, 1.0, 0.5, 0.2999], [0.25, 0.75, 0.099, 0.1]])
    cb = oracle.quantise(C, 0.25)
    assert cb.tolist() == [[0, 4, 2, 1], [1, 3, 0, 0]]
    cb = oracle.quantise(C, 0.1)
    # the FP64 number 0.1 is slightly above 1/10, so 10 * 0.1 > 1.0 exactly:
    # floor(1.0 / 0.1) = 9 (exact quotient 9.99...), likewise 0.5 -> 4.
    assert cb.tolist() == [[0, 9, 4, 2], [2, 7, 0, 1]]


def exact_floor(c, eps):
    return math.floor(Fraction(c) / Fraction(eps))


def test_quantise_is_exact_floor_everywhere():
    """Eq. (1) exactly: cb = floor of the exact rational quotient c/eps, for
    random costs and for costs placed on and next to multiples of eps."""
    g = np.random.default_rng(7)
    for eps in (0.1, 0.01, 0.005, 0.3, 1.0 / 3.0, 1.0 / 32766.5):
        K = int(math.floor(1.0 / eps))
        vals = list(g.random(400))
        ks = g.integers(0, K + 1, size=200)
        for k in ks:
            v = float(k) * eps                   # RN(k * eps): either side of k*eps
            for x in (v, np.nextafter(v, 0.0), np.nextafter(v, 2.0)):
                if 0.0 <= x <= 1.0:
                    vals.append(float(x))
        vals += [0.0, 1.0, 5e-324, np.nextafter(1.0, 0.0)]
        C = np.array(vals, dtype=np.float64).reshape(1, -1)
        cb = oracle.quantise(C, eps)
        want = [exact_floor(c, eps) for c in C[0]]
        assert cb[0].tolist() == want


def test_quantise_exact_floor_differs_from_rounded_division():
    """There are costs where floor(RN(c/eps)) overshoots the exact floor; the
    oracle follows Eq. (1) exactly there."""
    eps = 0.1
    hits = 0
    for k in range(1, 11):
        for x in (float(k) * eps, np.nextafter(float(k) * eps, 0.0)):
            if x <= 1.0 and math.floor(x / eps) != exact_floor(x, eps):
                hits += 1
                cb = oracle.quantise(np.array([[x]]), eps)
                assert cb[0, 0] == exact_floor(x, eps)
    assert hits > 0


def test_quantise_rejects_out_of_range():
    for bad in (-1e-300, 1.0000000000000002, np.nan, np.inf):
        C = np.zeros((2, 2))
        C[1, 1] = bad
        with pytest.raises(ValueError):
            oracle.quantise(C, 0.1)


def test_threshold():
    assert oracle.threshold(0.01, 10000) == 100
    assert oracle.threshold(0.1, 1000) == 100
    assert oracle.threshold(0.005, 10000) == 50
    assert oracle.threshold(0.3, 3) == 0
    assert oracle.threshold(0.5, 3) == 1


# -------------------------------------------------------------------------
# Hand-worked run (tests/golden/assign_3x3_hand.txt)
# -------------------------------------------------------------------------

def test_golden_hand_run():
    g = read_golden("assign_3x3_hand.txt")
    eps = float(g["eps"][0][0])
    C = np.array([[float(x) for x in row] for row in g["C"]])
    r = oracle.assign(C, eps, mode=oracle.MODE_CHECK)
    assert r["cbar"].tolist() == [[int(x) for x in row] for row in g["cbar"]]
    assert r["threshold"] == int(g["threshold"][0][0])
    assert r["stats"]["phases"] == int(g["phases"][0][0])
    assert r["stats"]["rounds"] == int(g["rounds"][0][0])
    assert r["row_to_col"].tolist() == [int(x) for x in g["row_to_col"][0]]
    assert r["col_to_row"].tolist() == [int(x) for x in g["col_to_row"][0]]
    assert r["y_row"].tolist() == [int(x) for x in g["y_row"][0]]
    assert r["y_col"].tolist() == [int(x) for x in g["y_col"][0]]
    assert r["cost"] == float(g["cost"][0][0])
    assert r["stats"]["violations"] == 0


# -------------------------------------------------------------------------
# Closed forms
# -------------------------------------------------------------------------

@pytest.mark.parametrize("n,k,eps", [(5, 0.55, 0.1), (7, 1.0, 0.25), (4, 0.0, 0.5), (9, 0.31, 0.05)])
def test_constant_costs(n, k, eps):
    """C == k: K = floor(k/eps) pure relabel phases, then one phase of n rounds
    in which b_i takes a_i (lowest-index proposal and acceptance)."""
    C = np.full((n, n), k)
    K = int(math.floor(k / eps))
    T = oracle.threshold(eps, n)
    assert T < n
    r = oracle.assign(C, eps, mode=oracle.MODE_CHECK)
    assert r["stats"]["phases"] == K + 1
    assert r["stats"]["rounds"] == n
    assert r["row_to_col"].tolist() == list(range(n))
    assert (r["y_row"] == K + 1).all()
    assert (r["y_col"] == -1).all()
    assert r["stats"]["violations"] == 0


@pytest.mark.parametrize("n", [1, 2, 6, 33])
def test_zero_diagonal(n):
    C = 1.0 - np.eye(n)
    r = oracle.assign(C, 0.1, mode=oracle.MODE_CHECK)
    assert r["row_to_col"].tolist() == list(range(n))
    assert r["stats"]["phases"] == 1 and r["stats"]["rounds"] == 1
    assert (r["y_col"] == -1).all() and (r["y_row"] == 1).all()
    assert r["cost"] == 0.0


@pytest.mark.parametrize("seed", range(4))
def test_zero_permutation(seed):
    n = 17
    pi = np.random.default_rng(seed).permutation(n)
    C = np.ones((n, n))
    C[np.arange(n), pi] = 0.0
    r = oracle.assign(C, 0.2)
    assert r["row_to_col"].tolist() == pi.tolist()
    assert r["stats"]["phases"] == 1
    assert r["cost"] == 0.0


def test_single_vertex():
    """n = 1: T = 0, the row relabels until y_b = cb + 1, then matches."""
    for c, eps in ((0.73, 0.1), (0.0, 0.3), (1.0, 0.25)):
        r = oracle.assign(np.array([[c]]), eps)
        K = int(math.floor(c / eps))
        assert r["stats"]["phases"] == K + 1
        assert r["y_row"][0] == K + 1 and r["y_col"][0] == -1
        assert r["row_to_col"][0] == 0


# -------------------------------------------------------------------------
# Bounds and invariants on random instances
# -------------------------------------------------------------------------

def _check_bounds(C, eps, r, opt=None):
    nB, nA = C.shape
    K = int(math.floor(1.0 / eps))
    T = r["threshold"]
    st = r["stats"]
    yb, ya = r["y_row"].astype(np.int64), r["y_col"].astype(np.int64)
    # perfect (row-complete) matching
    assert len(set(r["row_to_col"].tolist())) == nB
    assert (r["row_to_col"] >= 0).all()
    assert st["free_at_stop"] <= T
    # Lemma 3.2 (eps units): |y| <= floor(1/eps) + 2
    assert yb.max() <= K + 2 and -ya.min() <= K + 2
    # Lemma 3.3 made exact: the total dual magnitude grows by |B'| per phase.
    assert yb.sum() - ya.sum() - nB == st["sum_ni"]
    # Eq. (4) with the factor 2 the 2n vertices need; phase bound of Sec. 3.2.
    assert st["sum_ni"] <= nB * (2 * K + 3)
    assert st["phases"] <= oracle.phase_cap(eps, nB)
    # Lemma 3.1 dual certificate: L = eps (sum y - |B|) <= OPT(cbar) <= OPT(c),
    # and c(M) <= L + 2 eps |B| + T (completion edges cost at most 1).
    L = eps * (yb.sum() + ya.sum() - nB)
    assert r["cost"] <= L + 2 * eps * nB + T + 1e-9
    if opt is not None:
        assert L <= opt + 1e-9
        assert opt - 1e-9 <= r["cost"] <= opt + 3 * eps * nB + 1e-9
    return L


@pytest.mark.parametrize("seed", range(30))
def test_brute_force_bound_small(seed):
    g = np.random.default_rng(100 + seed)
    nB = int(g.integers(1, 8))
    nA = int(g.integers(nB, 8))
    C = rand_costs(seed, nB, nA, "uniform" if seed % 3 else "few")
    opt = brute_force(C)
    for eps in EPS_SET:
        r = oracle.assign(C, eps, mode=oracle.MODE_CHECK)
        assert r["stats"]["violations"] == 0
        L = _check_bounds(C, eps, r, opt)
        # L also bounds the rounded optimum (Lemma 3.1 with costs cbar).
        cbar_opt = brute_force(r["cbar"].astype(np.float64) * eps)
        assert L <= cbar_opt + 1e-9


@pytest.mark.parametrize("n,eps,sq", [(60, 0.1, True), (150, 0.05, False), (200, 0.01, False),
                                      (120, 0.005, False), (90, 0.3, True)])
def test_invariants_every_phase_and_hungarian_bound(n, eps, sq):
    C = W.assignment_sq_euclid_2d(n, n) if sq else W.assignment_euclid_2d(n, n)
    r = oracle.assign(C, eps, mode=oracle.MODE_CHECK)
    assert r["stats"]["violations"] == 0
    opt, _ = oracle.hungarian(C)
    _check_bounds(C, eps, r, opt)


@pytest.mark.parametrize("nB,nA", [(30, 45), (64, 200), (1, 9)])
def test_unbalanced(nB, nA):
    """Sec. 3.3: |B| <= |A|; stops at <= eps|B| free; Lemma 3.5 bound."""
    A, B = W.points_uniform(nA, nB, 2, 5)
    C = W.pairwise_cost(A, B, squared=False)
    for eps in (0.1, 0.02):
        r = oracle.assign(C, eps, mode=oracle.MODE_CHECK)
        assert r["stats"]["violations"] == 0
        opt, _ = oracle.hungarian(C)
        _check_bounds(C, eps, r, opt)


# -------------------------------------------------------------------------
# The round rule itself
# -------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_literal_rescan_equals_resume_pointer(seed):
    n = 70
    C = W.assignment_euclid_2d(n, seed) if seed % 2 else rand_costs(seed, n, n, "few")
    for eps in (0.1, 0.02):
        cb = oracle.quantise(C, eps)
        T = oracle.threshold(eps, n)
        r0 = oracle.assign_int(cb, T, mode=oracle.MODE_RESUME)
        r1 = oracle.assign_int(cb, T, mode=oracle.MODE_LITERAL)
        r2 = oracle.assign_int(cb, T, mode=oracle.MODE_REVERSE)
        for k in ("match_b", "match_a", "y_b", "y_a"):
            assert np.array_equal(r0[k], r1[k]) and np.array_equal(r0[k], r2[k])
        for k in ("phases", "rounds", "sum_ni"):
            assert r0["stats"][k] == r1["stats"][k] == r2["stats"][k]


@pytest.mark.parametrize("seed", range(6))
def test_evict_resume_equals_resume_pointer(seed):
    """Starting an evicted row's next scan after the column it lost changes
    no proposal (every earlier column stays inadmissible, Eq. 2 with growing
    keys): same matching, duals, phases and rounds, and never more entries
    examined.  The literal rescan, with every row starting at column 0,
    examines the most."""
    n = 90
    C = W.assignment_euclid_2d(n, seed) if seed % 2 else rand_costs(seed, n, n, "few")
    for eps in (0.1, 0.02, 0.005):
        cb = oracle.quantise(C, eps)
        T = oracle.threshold(eps, n)
        r0 = oracle.assign_int(cb, T, mode=oracle.MODE_RESUME)
        r1 = oracle.assign_int(cb, T, mode=oracle.MODE_EVICT_RESUME | oracle.MODE_CHECK)
        r2 = oracle.assign_int(cb, T, mode=oracle.MODE_EVICT_RESUME | oracle.MODE_REVERSE)
        for k in ("match_b", "match_a", "y_b", "y_a"):
            assert np.array_equal(r0[k], r1[k]) and np.array_equal(r0[k], r2[k])
        for k in ("phases", "rounds", "sum_ni"):
            assert r0["stats"][k] == r1["stats"][k] == r2["stats"][k]
        assert r1["stats"]["violations"] == 0
        assert r1["stats"]["scanned"] == r2["stats"]["scanned"] <= r0["stats"]["scanned"]
        r3 = oracle.assign_int(cb, T, mode=oracle.MODE_LITERAL)
        assert r0["stats"]["scanned"] <= r3["stats"]["scanned"]


def test_evict_resume_skips_entries_on_a_hand_case():
    """Two rows, two columns, eps = 0.5 (cb in {0, 1, 2}).  Row 0 takes column
    0 in phase 1 and loses it to row 1 in phase 2; in phase 3 row 0 starts
    at column 1 instead of 0, one entry fewer, with the same outcome."""
    C = np.array([[0.0, 0.0], [0.0, 1.0]])
    cb = oracle.quantise(C, 0.5)
    assert cb.tolist() == [[0, 0], [0, 2]]
    r0 = oracle.assign_int(cb, 0, mode=oracle.MODE_RESUME)
    r1 = oracle.assign_int(cb, 0, mode=oracle.MODE_EVICT_RESUME)
    for k in ("match_b", "match_a", "y_b", "y_a"):
        assert np.array_equal(r0[k], r1[k])
    assert r0["match_b"].tolist() == [1, 0]
    assert r0["stats"]["scanned"] - r1["stats"]["scanned"] >= 1


def test_sequential_greedy_is_valid_but_different():
    """The paper's own sequential greedy (Lemma 3.4) gives another valid run:
    same invariants and bounds, generally a different matching."""
    n = 80
    C = W.assignment_sq_euclid_2d(n, 3)
    eps = 0.1
    cb = oracle.quantise(C, eps)
    T = oracle.threshold(eps, n)
    rs = oracle.assign_int(cb, T, mode=oracle.MODE_SEQUENTIAL | oracle.MODE_CHECK)
    rr = oracle.assign_int(cb, T, mode=oracle.MODE_CHECK)
    assert rs["stats"]["violations"] == 0 and rr["stats"]["violations"] == 0
    assert not np.array_equal(rs["match_b"], rr["match_b"])


def test_cost_is_exactly_rounded_sum():
    C = W.assignment_euclid_2d(500, 1)
    r = oracle.assign(C, 0.05)
    exact = math.fsum(C[np.arange(500), r["row_to_col"]])
    assert abs(r["cost"] - exact) <= 1e-15 * exact


def test_float32_input_widened_exactly():
    C = W.assignment_euclid_2d(50, 2).astype(np.float32)
    r32 = oracle.assign(C, 0.05)
    r64 = oracle.assign(C.astype(np.float64), 0.05)
    assert np.array_equal(r32["row_to_col"], r64["row_to_col"])
    assert r32["cost"] == r64["cost"]


# -------------------------------------------------------------------------
# Another step I rule: seeded start columns (OR_MODE_OFFSET)
# -------------------------------------------------------------------------

def _splitmix64(x):
    """SplitMix64's output function (Steele, Lea, Flood, OOPSLA 2014)."""
    M = (1 << 64) - 1
    x = (x + 0x9E3779B97F4A7C15) & M
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & M
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & M
    return x ^ (x >> 31)


def _offset_rule_literal(cb, T):
    """Sec. 2.2 with the offset rule, written out in Python: in phase p
    every free b scans cyclically from column splitmix64(p << 32 | b) mod n_A
    and proposes to the first admissible column not taken in an earlier
    round; each column takes its lowest proposer; losers go on after the
    column they lost until they have seen every column once."""
    nB, nA = len(cb), len(cb[0])
    yb, ya = [1] * nB, [0] * nA
    mb, ma = [-1] * nB, [-1] * nA
    phases = rounds = 0
    while True:
        F = [b for b in range(nB) if mb[b] < 0]
        if len(F) <= T:
            break
        phases += 1
        pos = {b: _splitmix64((phases << 32) | b) % nA for b in F}
        seen = {b: 0 for b in F}
        taken, mate, act = set(), {b: -1 for b in F}, list(F)
        while True:
            prop = {}
            for b in act:
                while seen[b] < nA:
                    a = pos[b]
                    pos[b] = (a + 1) % nA
                    seen[b] += 1
                    if a not in taken and ya[a] + yb[b] == cb[b][a] + 1:
                        prop[b] = a
                        break
            if not prop:
                break
            rounds += 1
            win = {}
            for b, a in prop.items():
                win[a] = min(win.get(a, nB), b)
            act = [b for b, a in prop.items() if win[a] != b]
            for a, b in win.items():
                mate[b] = a
                taken.add(a)
            if not act:
                break
        for b in F:
            a = mate[b]
            if a >= 0:
                if ma[a] >= 0:
                    mb[ma[a]] = -1
                ma[a], mb[b] = b, a
        for b in F:
            if mate[b] >= 0:
                ya[mate[b]] -= 1
            else:
                yb[b] += 1
    return mb, ma, yb, ya, phases, rounds


@pytest.mark.parametrize("seed", range(8))
def test_offset_rule_equals_literal_restatement(seed):
    g = np.random.default_rng(seed)
    n = int(g.integers(2, 9))
    C = rand_costs(seed, n, n, "few" if seed % 2 else "uniform")
    for eps in (0.5, 0.2, 0.1):
        cb = oracle.quantise(C, eps)
        T = oracle.threshold(eps, n)
        r = oracle.assign_int(cb, T, mode=oracle.MODE_OFFSET)
        mb, ma, yb, ya, ph, rd = _offset_rule_literal(cb.tolist(), T)
        assert r["match_b"].tolist() == mb and r["match_a"].tolist() == ma
        assert r["y_b"].tolist() == yb and r["y_a"].tolist() == ya
        assert r["stats"]["phases"] == ph and r["stats"]["rounds"] == rd


@pytest.mark.parametrize("n,eps,sq", [(60, 0.1, True), (150, 0.02, False), (300, 0.005, True)])
def test_offset_rule_invariants_and_bound(n, eps, sq):
    """Any maximal matching per phase keeps Lemma 2.1, (I1)/(I2) and the
    3 eps n bound (Sec. 2.1); the offset rule is one."""
    C = W.assignment_sq_euclid_2d(n, 3) if sq else W.assignment_euclid_2d(n, 3)
    r = oracle.assign(C, eps, mode=oracle.MODE_OFFSET | oracle.MODE_CHECK)
    assert r["stats"]["violations"] == 0
    opt, _ = oracle.hungarian(C)
    assert opt - 1e-12 <= r["cost"] <= opt + 3 * eps * n + 1e-12


def test_offset_rule_breaks_the_round_convoy():
    """Where most edges are admissible (large eps) the lowest-index rule
    sends every loser to the same next columns and needs many rounds; start
    columns spread the proposals.  Recorded on the MNIST-shaped workload."""
    A, B = W.mnist_shaped_pair(400, 3)
    C = W.l1_cost(A, B)
    cb = oracle.quantise(C, 0.75)
    T = oracle.threshold(0.75, 400)
    low = oracle.assign_int(cb, T)["stats"]
    off = oracle.assign_int(cb, T, mode=oracle.MODE_OFFSET)["stats"]
    assert low["phases"] == off["phases"] == 1
    assert off["rounds"] * 4 < low["rounds"]


@pytest.mark.parametrize("mode", [0, 32])
def test_parallel_scans_change_nothing(mode):
    """OR_MODE_PARALLEL (the scans of a round on all host cores, for timing)
    gives the same matching, duals and counters as the serial oracle."""
    C = W.assignment_euclid_2d(700, 12)
    for eps in (0.1, 0.01):
        r0 = oracle.assign(C, eps, mode=mode)
        r1 = oracle.assign(C, eps, mode=mode | oracle.MODE_PARALLEL)
        for k in ("row_to_col", "col_to_row", "y_row", "y_col"):
            assert np.array_equal(r0[k], r1[k])
        assert r0["stats"] == r1["stats"] and r0["cost"] == r1["cost"]


def test_state_checker_catches_planted_mistakes():
    """or_check_state (behind the per-phase invariant mode) is not vacuous:
    a final state passes, and each planted mistake is reported: a matched
    pair whose duals no longer sum to cbar (Eq. 3), a pair over cbar + 1
    (Eq. 2), a negative row dual or a free column with a nonzero dual (I1),
    and match arrays that disagree."""
    C = W.assignment_euclid_2d(30, 3)
    eps = 0.1
    cb = oracle.quantise(C, eps)
    r = oracle.assign_int(cb, oracle.threshold(eps, 30))
    mb, ma, yb, ya = (r[k].copy() for k in ("match_b", "match_a", "y_b", "y_a"))
    assert oracle.check_state(cb, mb, ma, yb, ya) == 0
    b = int(np.flatnonzero(mb >= 0)[0])
    a = int(mb[b])

    def bad(**kw):
        s = dict(match_b=mb.copy(), match_a=ma.copy(), y_b=yb.copy(), y_a=ya.copy())
        for k, f in kw.items():
            f(s[k])
        return oracle.check_state(cb, s["match_b"], s["match_a"], s["y_b"], s["y_a"])

    assert bad(y_b=lambda v: v.__setitem__(b, v[b] + 1)) > 0
    a2 = next(x for x in range(cb.shape[1]) if x != a)
    assert bad(y_a=lambda v: v.__setitem__(a2, cb[b, a2] + 2 - yb[b])) > 0
    assert bad(y_b=lambda v: v.__setitem__(b, -1)) > 0
    free_a = np.flatnonzero(ma < 0)
    if free_a.size:
        assert bad(y_a=lambda v: v.__setitem__(int(free_a[0]), -1)) > 0
    assert bad(match_a=lambda v: v.__setitem__(a, -1)) > 0


# -------------------------------------------------------------------------
# A third step I rule: Israeli and Itai's randomized maximal matching
# (Sec. 3.2, parallel efficiency), OR_MODE_ISRAELI_ITAI
# -------------------------------------------------------------------------

_COL = 1 << 24


def _ii_draw(step, phase, it, u, v):
    """Three SplitMix64 rounds: over (step, phase, iteration), then the
    vertex id, then the other end."""
    x = _splitmix64(((step << 56) ^ (phase << 28) ^ it) & ((1 << 64) - 1))
    x = _splitmix64(x ^ u)
    return _splitmix64(x ^ v)


def _ii_key(step, phase, it, u, v):
    return ((_ii_draw(step, phase, it, u, v) >> 24) << 24) | (v & 0xFFFFFF)


def test_israeli_itai_key_equals_its_definition():
    g = np.random.default_rng(5)
    for _ in range(200):
        args = [int(g.integers(1, 4)), int(g.integers(1, 1 << 20)), int(g.integers(1, 5000)),
                int(g.integers(0, 1 << 25)), int(g.integers(0, 1 << 24))]
        assert oracle.ii_key(*args) == _ii_key(*args)


def _israeli_itai_literal(cb, T):
    """Sec. 2.2 with step I by Israeli-Itai rounds, written out in Python.
    Per iteration on the admissible graph of the live free rows and the
    columns not yet in M': (1) each vertex with an edge points to the
    neighbour of least key; (2) each vertex pointed at keeps the pointer of
    least key; (3) each vertex picks one of its kept edges (the one it points
    along, the one kept pointing at it; a coin bit when both), and an edge
    picked at both ends joins M'.  Rows without an edge drop out."""
    nB, nA = len(cb), len(cb[0])
    yb, ya = [1] * nB, [0] * nA
    mb, ma = [-1] * nB, [-1] * nA
    phases = rounds = 0
    while True:
        F = [b for b in range(nB) if mb[b] < 0]
        if len(F) <= T:
            break
        phases += 1
        live, taken, mate = set(F), set(), {b: -1 for b in F}
        it = 0
        while True:
            it += 1
            edges = {b: [a for a in range(nA) if a not in taken and ya[a] + yb[b] == cb[b][a] + 1]
                     for b in sorted(live)}
            live = {b for b in live if edges[b]}
            if not live:
                break
            rounds += 1
            out_r = {b: min(edges[b], key=lambda a: _ii_key(1, phases, it, b, a)) for b in live}
            nbr_c = {}
            for b in live:
                for a in edges[b]:
                    nbr_c.setdefault(a, []).append(b)
            out_c = {a: min(bs, key=lambda b: _ii_key(1, phases, it, _COL + a, b)) for a, bs in nbr_c.items()}
            in_c, in_r = {}, {}
            for b, a in out_r.items():
                if a not in in_c or _ii_key(2, phases, it, _COL + a, b) < _ii_key(2, phases, it, _COL + a, in_c[a]):
                    in_c[a] = b
            for a, b in out_c.items():
                if b not in in_r or _ii_key(2, phases, it, b, a) < _ii_key(2, phases, it, b, in_r[b]):
                    in_r[b] = a

            def pick(u, out, inn):
                if out is not None and inn is not None:
                    return inn if _ii_draw(3, phases, it, u, 0) & 1 else out
                return out if out is not None else inn

            pr = {b: pick(b, out_r[b] if in_c.get(out_r[b]) == b else None, in_r.get(b)) for b in live}
            pc = {a: pick(_COL + a, out_c[a] if in_r.get(out_c[a]) == a else None, in_c.get(a))
                  for a in nbr_c}
            for b in sorted(live):
                a = pr[b]
                if a is not None and pc.get(a) == b:
                    mate[b] = a
                    taken.add(a)
            live -= {b for b in live if mate[b] >= 0}
        for b in F:
            a = mate[b]
            if a >= 0:
                if ma[a] >= 0:
                    mb[ma[a]] = -1
                ma[a], mb[b] = b, a
        for b in F:
            if mate[b] >= 0:
                ya[mate[b]] -= 1
            else:
                yb[b] += 1
    return mb, ma, yb, ya, phases, rounds


@pytest.mark.parametrize("seed", range(8))
def test_israeli_itai_equals_literal_restatement(seed):
    g = np.random.default_rng(100 + seed)
    n = int(g.integers(2, 10))
    C = rand_costs(seed, n, n + int(g.integers(0, 3)), "few" if seed % 2 else "uniform")
    for eps in (0.5, 0.2, 0.1):
        cb = oracle.quantise(C, eps)
        T = oracle.threshold(eps, C.shape[0])
        r = oracle.assign_int(cb, T, mode=oracle.MODE_ISRAELI_ITAI)
        mb, ma, yb, ya, ph, rd = _israeli_itai_literal(cb.tolist(), T)
        assert r["match_b"].tolist() == mb and r["match_a"].tolist() == ma
        assert r["y_b"].tolist() == yb and r["y_a"].tolist() == ya
        assert r["stats"]["phases"] == ph and r["stats"]["rounds"] == rd


@pytest.mark.parametrize("n,eps,sq", [(60, 0.1, True), (150, 0.02, False), (300, 0.005, True)])
def test_israeli_itai_invariants_and_bound(n, eps, sq):
    """Every phase leaves a maximal M' (a relabelled row with an admissible
    untaken column would break Eq. 2, which the per-phase check sees),
    (I1)/(I2) and Lemma 2.1 hold, and the cost is within 3 eps n of the
    optimum (Sec. 2.1)."""
    C = W.assignment_sq_euclid_2d(n, 3) if sq else W.assignment_euclid_2d(n, 3)
    r = oracle.assign(C, eps, mode=oracle.MODE_ISRAELI_ITAI | oracle.MODE_CHECK)
    assert r["stats"]["violations"] == 0
    opt, _ = oracle.hungarian(C)
    assert opt - 1e-12 <= r["cost"] <= opt + 3 * eps * n + 1e-12


def test_israeli_itai_rounds_stay_logarithmic():
    """Where most edges are admissible (MNIST-shaped, eps = 0.75) the
    lowest-index rule needs hundreds of rounds in its one phase; the
    randomized rule stays within a few times log2 n (Sec. 3.2)."""
    A, B = W.mnist_shaped_pair(400, 3)
    C = W.l1_cost(A, B)
    cb = oracle.quantise(C, 0.75)
    T = oracle.threshold(0.75, 400)
    low = oracle.assign_int(cb, T)["stats"]
    ii = oracle.assign_int(cb, T, mode=oracle.MODE_ISRAELI_ITAI)["stats"]
    assert ii["phases"] == 1
    assert ii["rounds"] <= 4 * np.log2(400) < low["rounds"]


# -------------------------------------------------------------------------
# Step I without rounds: displacement chains give the sequential greedy
# -------------------------------------------------------------------------

def _displacement_run(cb, T, rng):
    """Sec. 2.2 with step I run as concurrent chains and no rounds: every
    free row scans its columns in order for an admissible one; a column is
    held by the lowest row that reached it in this phase, so a row passes a
    column held by a lower row and takes one held by a higher row, whose row
    then goes on scanning after that column.  The chains advance one column
    at a time in the order `rng` draws.  A row evicted from M starts its next
    scan after the column it lost, as in the evict-resume rule.  Steps II and
    III are those of Sec. 2.2."""
    nB, nA = cb.shape
    y_b, k = [1] * nB, [0] * nA
    partner, match_b, start = [-1] * nA, [-1] * nB, [0] * nB
    phases = 0
    while True:
        free = [b for b in range(nB) if match_b[b] < 0]
        if len(free) <= T:
            break
        phases += 1
        held = {}
        active = [(b, start[b]) for b in free]
        for b in free:
            start[b] = 0
        while active:
            i = int(rng.integers(len(active)))
            b, a = active[i]
            if a >= nA:
                active.pop(i)
                continue
            if cb[b, a] + k[a] == y_b[b] - 1 and held.get(a, nB) > b:
                h = held.get(a)
                held[a] = b
                if h is None:
                    active.pop(i)
                else:
                    active[i] = (h, a + 1)
                continue
            active[i] = (b, a + 1)
        mate = {b: a for a, b in held.items()}
        for a, b in held.items():
            old = partner[a]
            if old >= 0:
                match_b[old] = -1
                start[old] = a + 1
            partner[a], match_b[b] = b, a
            k[a] += 1
        for b in free:
            if b not in mate:
                y_b[b] += 1
    return np.array(match_b), np.array(y_b), -np.array(k), phases


@pytest.mark.parametrize("seed", range(8))
def test_displacement_chains_give_the_sequential_greedy(seed):
    """Whatever order the chains advance in, each phase ends with the
    matching M' of the paper's sequential greedy (Sec. 3.2: rows in index
    order, each takes its first admissible column not yet in M'), so the
    whole run equals OR_MODE_SEQUENTIAL: matching, both duals and phases.
    Few distinct costs make many rows compete for the same columns."""
    g = np.random.default_rng(seed)
    nB = int(g.integers(6, 30))
    nA = nB + int(g.integers(0, 6))
    eps = (0.1, 0.25, 0.05)[seed % 3]
    C = rand_costs(seed, nB, nA, "few" if seed % 2 else "uniform")
    cb = oracle.quantise(C, eps)
    T = oracle.threshold(eps, nB)
    ref = oracle.assign_int(cb, T, mode=oracle.MODE_SEQUENTIAL)
    for order in range(3):
        mb, yb, ya, phases = _displacement_run(cb, T, np.random.default_rng(100 * seed + order))
        assert np.array_equal(mb, ref["match_b"])
        assert np.array_equal(yb, ref["y_b"])
        assert np.array_equal(ya, ref["y_a"])
        assert phases == ref["stats"]["phases"] == ref["stats"]["rounds"]


def test_displacement_chains_differ_from_the_round_rule():
    """The chains are not the lowest-index round rule: on the MNIST-shaped
    costs at eps = 0.75 the two rules pick different matchings."""
    A, B = W.mnist_shaped_pair(60, 2)
    C = W.l1_cost(A, B)
    cb = oracle.quantise(C, 0.75)
    T = oracle.threshold(0.75, 60)
    mb, _, _, _ = _displacement_run(cb, T, np.random.default_rng(0))
    assert not np.array_equal(mb, oracle.assign_int(cb, T)["match_b"])
