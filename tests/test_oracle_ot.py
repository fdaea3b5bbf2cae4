"""Pins for the OT oracle (Sec. 4), CPU only: one copy per vertex reduces to
the assignment routine; invariants and the two-cluster lemma on the implied
copy state; plan feasibility; the additive bound against an exact LP (scipy
HiGHS); hand-computed mass quantisation."""
import numpy as np
import pytest

import oracle
from oracle import ot as O
from paper_2203_03732_gb300 import workloads as W


def lp_opt(C, nu, mu):
    from scipy.optimize import linprog
    nB, nA = C.shape
    A_eq = np.zeros((nB, nB * nA))
    for b in range(nB):
        A_eq[b, b * nA:(b + 1) * nA] = 1
    A_ub = np.zeros((nA, nB * nA))
    for a in range(nA):
        A_ub[a, a::nA] = 1
    r = linprog(C.ravel(), A_ub=A_ub, b_ub=mu, A_eq=A_eq, b_eq=nu, bounds=(0, None), method="highs")
    assert r.status == 0
    return r.fun


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("eps", [0.1, 0.02])
def test_unit_copies_equal_assignment(seed, eps):
    """With one copy per vertex the cluster phases are the Sec. 2.2 routine."""
    n = 60
    C = W.assignment_euclid_2d(n, seed)
    cb = oracle.quantise(C, eps)
    T = oracle.threshold(eps, n)
    a = oracle.assign_int(cb, T)
    r = O.cluster_int(cb, np.ones(n, np.int32), np.ones(n, np.int32), T)
    assert r["stats"]["phases"] == a["stats"]["phases"]
    assert r["stats"]["rounds"] == a["stats"]["rounds"]
    assert r["stats"]["free_at_stop"] == a["stats"]["free_at_stop"]
    plan = r["plan_lo"] + r["plan_hi"]
    mb = np.where(plan.sum(1) > 0, plan.argmax(1), -1)
    assert np.array_equal(mb, a["match_b"])
    assert np.array_equal(r["F"], a["y_b"])
    assert np.array_equal(-r["kmin"], a["y_a"])


def copy_state_check(r, cb):
    """(I1)/(I2) and Lemma 4.1 on the copy instance the cluster state stands
    for: free supply copies of b have dual F_b; a matched copy in plan_lo /
    plan_hi at (b, a) has dual cbar + kmin_a / cbar + kmin_a + 1; a's copies
    have keys kmin_a (clo of them) and kmin_a + 1 (chi)."""
    F, f, kmin, clo, chi = r["F"], r["f"], r["kmin"], r["clo"], r["chi"]
    plo, phi = r["plan_lo"], r["plan_hi"]
    nB, nA = cb.shape
    assert (r["S"] == f + plo.sum(1) + phi.sum(1)).all()
    assert (phi.sum(0) == chi).all()
    assert ((kmin == 0) | (plo.sum(0) == clo)).all()
    assert ((kmin >= 1) | (plo.sum(0) == 0)).all()
    for b in range(nB):
        duals = set()
        if f[b] > 0:
            duals.add(int(F[b]))
        for a in range(nA):
            if plo[b, a]:
                duals.add(int(cb[b, a] + kmin[a]))
            if phi[b, a]:
                duals.add(int(cb[b, a] + kmin[a] + 1))
        if not duals:
            continue
        assert max(duals) <= F[b]               # raise rule: F_b is the largest
        if plo[b].sum() + phi[b].sum() > 0:
            assert max(duals) - min(duals) <= 1  # Lemma 4.1: two clusters
        # Eq. (2) for every copy of b against a's lowest key (its worst case);
        # a column without copies constrains nothing
        has = (clo + chi) > 0
        for y in duals:
            assert (y - kmin[has] <= cb[b][has] + 1).all()


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("eps", [0.2, 0.1, 0.05])
def test_invariants_plan_and_bound(seed, eps):
    nB, nA = (12, 15) if seed % 2 else (18, 18)
    C, nu, mu = W.ot_euclid_2d(nB, nA, 100 + seed)
    r = O.ot(C, nu, mu, eps, mode=oracle.MODE_CHECK)
    assert r["stats"]["violations"] == 0
    copy_state_check(r, r["cbar"])
    assert r["stats"]["free_at_stop"] <= r["T"]
    m = r["mass"]
    assert (m >= 0).all()
    assert np.abs(m.sum(1) - nu).max() <= 1e-12
    assert (m.sum(0) - mu).max() <= 1e-12
    opt = lp_opt(C, nu, mu)
    assert opt - 1e-9 <= r["cost"] <= opt + 3.5 * eps


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("eps", [0.1, 0.02])
def test_returned_duals_are_feasible(seed, eps):
    """What the OT form returns as duals (F_b per supply, kmin and the two
    cluster counts per demand) satisfies Eq. 2 on its own: every supply's
    dual F_b plus the highest dual among a demand's copies is at most
    cbar + 1 (units of eps), including supplies with no free copy left."""
    C, nu, mu = W.ot_euclid_2d(90 + 13 * seed, 70 + 29 * seed, 300 + seed)
    r = O.ot(C, nu, mu, eps)
    F = r["F"].astype(np.int64)
    kmin = r["kmin"].astype(np.int64)
    top = np.where(r["clo"] > 0, -kmin, -kmin - 1)
    assert not (F[:, None] + top[None, :] > r["cbar"].astype(np.int64) + 1).any()
    # the copy with the top dual of a demand with copies exists
    assert ((r["clo"] + r["chi"]) > 0).any()


def test_returned_duals_with_zero_masses():
    """Zero masses on both sides: a demand of mass 0 has D_a = 0 copies
    (Sec. 4) and so no dual to check; Eq. 2 holds between every supply's F_b
    and the highest dual of every demand that has copies."""
    C, nu, mu = W.ot_euclid_2d(40, 50, 3)
    nu = nu.copy()
    nu[[1, 7]] = 0.0
    nu /= nu.sum()
    mu = mu.copy()
    mu[[0, 4, 49]] = 0.0
    mu /= mu.sum()
    r = O.ot(C, nu, mu, 0.05)
    has = (r["clo"] + r["chi"]) > 0
    assert not has[[0, 4, 49]].any() and has.sum() == 47
    F = r["F"].astype(np.int64)
    kmin = r["kmin"].astype(np.int64)
    top = np.where(r["clo"] > 0, -kmin, -kmin - 1)
    assert not ((F[:, None] + top[None, :] > r["cbar"].astype(np.int64) + 1) & has[None, :]).any()


def test_theta_and_counts_by_hand():
    # n = 3, eps = 0.5: theta = 24; supplies 0.5/0.25/0.25 -> 12/6/6 copies,
    # demands 1/3 each -> ceil(24/3) = 8 copies.
    assert O.theta(3, 3, 0.5) == 24.0
    S, D = O.counts([0.5, 0.25, 0.25], [1 / 3, 1 / 3, 1 / 3], 0.5)
    assert S.tolist() == [12, 6, 6]
    assert D.tolist() == [8, 8, 8]
    # rectangular: n = max(2, 5) = 5, eps = 0.4 -> theta = 50
    S, D = O.counts([0.7, 0.3], [0.2] * 5, 0.4)
    assert S.tolist() == [35, 15] and D.tolist() == [10] * 5


def test_single_pair():
    C = np.array([[0.37]])
    r = O.ot(C, [1.0], [1.0], 0.1)
    assert r["mass"][0, 0] == 1.0
    assert abs(r["cost"] - 0.37) < 1e-15


def test_zero_masses_and_concentrated_supply():
    C, nu, mu = W.ot_euclid_2d(8, 10, 7)
    nu = np.zeros(8)
    nu[3] = 1.0
    mu = mu.copy()
    mu[[0, 4]] = 0.0
    mu /= mu.sum()
    r = O.ot(C, nu, mu, 0.1, mode=oracle.MODE_CHECK)
    assert r["stats"]["violations"] == 0
    assert np.abs(r["mass"].sum(1) - nu).max() <= 1e-12
    assert (r["mass"][:, [0, 4]] == 0).all()
    assert r["cost"] <= lp_opt(C, nu, mu) + 3.5 * 0.1


def test_north_west_by_hand():
    """The fix-up alone (no matched copies): the north-west corner rule on
    dyadic masses, tables worked by hand.  Every amount is a whole number of
    2^-62 units below 2^53 of them, so each is exact in FP64."""
    C = np.array([[0.5, 0.25, 1.0], [0.125, 0.75, 0.5], [1.0, 0.0, 0.25]])
    z = np.zeros((3, 3), np.int32)
    m, c = O.fixup(C, [0.5, 0.25, 0.25], [0.25, 0.5, 0.25], 10.0, z)
    assert np.array_equal(m, [[0.25, 0.25, 0], [0, 0.25, 0], [0, 0, 0.25]])
    assert c == 0.25 * 0.5 + 0.25 * 0.25 + 0.25 * 0.75 + 0.25 * 0.25
    # an empty supply and an empty demand; supply 0 and demand 0 end together
    C4 = np.full((3, 4), 0.5)
    m, _ = O.fixup(C4, [0.25, 0.0, 0.75], [0.25, 0.25, 0.0, 0.5], 10.0, np.zeros((3, 4), np.int32))
    assert np.array_equal(m, [[0.25, 0, 0, 0], [0, 0, 0, 0], [0, 0.25, 0, 0.5]])
    # capacity runs out first: the last supply keeps its remainder
    m, _ = O.fixup(np.full((3, 1), 0.5), [0.25, 0.5, 0.25], [0.5], 10.0, np.zeros((3, 1), np.int32))
    assert np.array_equal(m, [[0.25], [0.25], [0.0]])


def test_north_west_after_matched_and_trimmed_copies():
    """Matched copies first (mass = count / theta), then the residuals.
    theta = 4.  Diagonal copies: each pair holds 1/4 and the walk adds the
    remaining 1/4 to the same pair.  Column 0 over-filled (2/4 + 1/4 > 1/2):
    the excess 1/4 leaves the highest supplier, b = 1, whose remainder 1/2
    then goes to column 1."""
    C = np.array([[0.5, 0.25], [0.125, 0.75]])
    m, _ = O.fixup(C, [0.5, 0.5], [0.5, 0.5], 4.0, np.array([[1, 0], [0, 1]], np.int32))
    assert np.array_equal(m, [[0.5, 0], [0, 0.5]])
    m, _ = O.fixup(C, [0.5, 0.5], [0.5, 0.5], 4.0, np.array([[2, 0], [1, 0]], np.int32))
    assert np.array_equal(m, [[0.5, 0], [0, 0.5]])


@pytest.mark.parametrize("seed", range(4))
def test_north_west_staircase_and_exact_units(seed):
    """On random masses the walk's entries form a staircase (b and a never
    decrease, one of them increases at each entry); on masses that are
    multiples of 2^-40 every supply's row sums to its mass exactly (sums of
    the FP64 entries taken in exact rational arithmetic)."""
    from fractions import Fraction
    g = np.random.Generator(np.random.PCG64(seed))
    nB, nA = 37 + seed, 29 + 3 * seed
    C = g.random((nB, nA))
    z = np.zeros((nB, nA), np.int32)
    nu, mu = g.exponential(size=nB), g.exponential(size=nA)
    nu /= nu.sum()
    mu /= mu.sum()
    m, _ = O.fixup(C, nu, mu, 1.0, z)
    bs, as_ = np.nonzero(m)  # row-major: b ascending, then a ascending
    assert (np.diff(bs) >= 0).all() and (np.diff(as_) >= 0).all()
    assert ((np.diff(bs) > 0) | (np.diff(as_) > 0)).all()
    assert np.abs(m.sum(1) - nu).max() <= 1e-15 and (m.sum(0) - mu).max() <= 1e-15
    q = lambda x: np.floor(x * 2.0 ** 40) / 2.0 ** 40
    nu_d, mu_d = q(nu), q(mu)
    mu_d[-1] += sum(Fraction(v) for v in nu_d) - sum(Fraction(v) for v in mu_d)  # equal totals
    m, _ = O.fixup(C, nu_d, mu_d, 1.0, z)
    for b in range(nB):
        assert sum(Fraction(v) for v in m[b]) == Fraction(nu_d[b])
    for a in range(nA):
        assert sum(Fraction(v) for v in m[:, a]) == Fraction(mu_d[a])


def test_counts_refuses_masses_that_do_not_sum_to_one():
    """A mass of 2 or more, or a side summing to more than 1.5, is refused;
    sums just below 1.5 pass."""
    with pytest.raises(ValueError):
        O.counts([1.0, 0.6], [0.8, 0.2], 0.5)
    with pytest.raises(ValueError):
        O.counts([0.5, 0.5], [0.5, 1.0], 0.5)
    with pytest.raises(ValueError):
        O.counts([2.0], [1.0], 0.5)
    S, D = O.counts([0.75, 0.74], [1.0], 0.5)  # theta = 4 * 2 / 0.5 = 16
    assert S.tolist() == [12, 11] and D.tolist() == [16]


@pytest.mark.parametrize("seed", range(3))
def test_expanded_form_with_unit_supply_copies_is_the_assignment_routine(seed):
    """One copy per supply vertex, each demand vertex split into 1-3 unit
    copies: the expanded form is Sec. 2.2 on the column-repeated costs, so
    the C assignment oracle gives the same matching, duals, phases and
    rounds."""
    from oracle.ot_expanded import ot_expanded
    g = np.random.Generator(np.random.PCG64(100 + seed))
    n, eps = 12, 0.1
    C = W.assignment_euclid_2d(n, seed, n_a=n + 3)
    cb = oracle.quantise(C, eps)
    D = g.integers(1, 4, size=n + 3)
    T = oracle.threshold(eps, n)
    e = ot_expanded(cb, np.ones(n, int), D, T)
    a = oracle.assign_int(np.repeat(cb, D, axis=1), T)
    assert e["phases"] == a["stats"]["phases"] and e["rounds"] == a["stats"]["rounds"]
    assert e["match"] == a["match_b"].tolist()
    assert e["y_sup"] == a["y_b"].tolist() and e["y_dem"] == a["y_a"].tolist()


SHAPES = [(3, 3, 0.5), (4, 3, 0.4), (3, 5, 0.5), (5, 5, 0.6)]


@pytest.mark.parametrize("seed", range(5))
def test_expanded_form_invariants_and_bounds(seed):
    """Sec. 4 written copy by copy on tiny instances: eps-feasibility on the
    copies (Eqs. 2 and 3), the raise invariant, the stop rule, and the plan
    after the fix-up feasible and within 3.5 eps of the exact LP optimum."""
    from oracle.ot_expanded import copy_violations, ot_expanded
    for nB, nA, eps in SHAPES:
        C, nu, mu = W.ot_euclid_2d(nB, nA, seed)
        cb = oracle.quantise(C, eps)
        S, D = O.counts(nu, mu, eps)
        T = int(np.floor(eps * S.sum()))
        e = ot_expanded(cb, S, D, T, O.ot_phase_cap(eps, int(S.sum())))
        assert copy_violations(e, cb) == 0
        assert e["free"] <= T
        mass, cost = O.fixup(C, nu, mu, O.theta(nB, nA, eps), e["counts"].astype(np.int32))
        assert np.abs(mass.sum(1) - nu).max() <= 1e-12 and (mass.sum(0) - mu).max() <= 1e-12
        assert cost <= lp_opt(C, nu, mu) + 3.5 * eps + 1e-12


def test_cluster_and_expanded_forms_mostly_agree():
    """The cluster oracle grants a vertex's proposal as many copies as are
    available and evicts from the highest supplier; the expanded form
    proposes and evicts copy by copy.  Both are maximal matchings of the copy
    graph, so they may differ, but on these 120 seeded tiny instances they
    give the same phases and matched-copy counts 108 times; a change to
    either that breaks the copy semantics shows up as a drop."""
    from oracle.ot_expanded import ot_expanded
    agree = 0
    for seed in range(30):
        for nB, nA, eps in SHAPES:
            C, nu, mu = W.ot_euclid_2d(nB, nA, seed)
            cb = oracle.quantise(C, eps)
            S, D = O.counts(nu, mu, eps)
            T = int(np.floor(eps * S.sum()))
            cap = O.ot_phase_cap(eps, int(S.sum()))
            r = O.cluster_int(cb, S, D, T, cap=cap)
            e = ot_expanded(cb, S, D, T, cap)
            agree += (r["stats"]["phases"] == e["phases"]
                      and np.array_equal(r["plan_lo"] + r["plan_hi"], e["counts"]))
    assert agree >= 100


@pytest.mark.parametrize("n,eps,seed", [(64, 0.5, 0), (128, 0.25, 2), (32, 0.125, 4), (16, 0.0625, 5),
                                        (64, 0.03125, 6)])
def test_one_copy_per_vertex_is_the_assignment_solve(n, eps, seed):
    """Masses 1/theta (theta = 4n/eps a power of two, so they are exact):
    every vertex is one copy, the cluster phases are Sec. 2.2's, and the
    fix-up routes the free supplies' masses north-west, i.e. the k-th free
    row to the k-th free column, which is the assignment's completion.  The
    whole OT solve then equals the assignment solve: plan = permutation /
    theta, the same duals, phases and rounds, cost / theta."""
    th = O.theta(n, n, eps)
    assert th == 2.0 ** round(np.log2(th))
    C = W.assignment_euclid_2d(n, seed)
    nu = np.full(n, 1.0 / th)
    r = O.ot(C, nu, nu.copy(), eps)
    a = oracle.assign(C, eps)
    assert set(r["S"].tolist()) == {1} and set(r["D"].tolist()) == {1}
    plan = np.zeros((n, n))
    plan[np.arange(n), a["row_to_col"]] = 1.0 / th
    assert np.array_equal(r["mass"], plan)
    assert np.array_equal(r["F"], a["y_row"]) and np.array_equal(-r["kmin"], a["y_col"])
    assert r["stats"]["phases"] == a["stats"]["phases"] and r["stats"]["rounds"] == a["stats"]["rounds"]
    assert abs(r["cost"] * th - a["cost"]) <= 1e-12 * a["cost"]


def test_copy_checker_catches_planted_mistakes():
    """The expanded form's checker is not vacuous: a matched pair off by one
    in its dual sum, a demand copy's dual raised above 0, a free supply copy
    below its siblings' dual, and a non-matched pair over cbar + 1 are each
    reported."""
    import copy
    from oracle.ot_expanded import copy_violations, ot_expanded
    C, nu, mu = W.ot_euclid_2d(4, 3, 1)
    eps = 0.4
    cb = oracle.quantise(C, eps)
    S, D = O.counts(nu, mu, eps)
    T = int(np.floor(eps * S.sum()))
    e = ot_expanded(cb, S, D, T)
    assert copy_violations(e, cb) == 0
    i = next(k for k, j in enumerate(e["match"]) if j >= 0)
    bad = copy.deepcopy(e)
    bad["y_sup"][i] += 1  # matched pair: sum no longer cbar
    assert copy_violations(bad, cb) > 0
    bad = copy.deepcopy(e)
    bad["y_dem"][e["match"][i]] = 1  # a demand dual above 0
    assert copy_violations(bad, cb) > 0
    free = [k for k, j in enumerate(e["match"]) if j < 0]
    if free:
        bad = copy.deepcopy(e)
        bad["y_sup"][free[0]] -= 1  # below its siblings (raise invariant)
        assert copy_violations(bad, cb) > 0
    bad = copy.deepcopy(e)
    j0 = next(j for j in range(len(e["dem"])) if j != e["match"][i])
    bad["y_dem"][j0] = cb[e["sup"][i]][e["dem"][j0]] + 2 - bad["y_sup"][i]  # over cbar + 1
    assert copy_violations(bad, cb) > 0
