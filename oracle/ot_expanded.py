"""Sec. 4 on the copy instance itself, written out with every copy
materialised: test infrastructure only, pure Python loops, for tiny inputs.

Every supply b becomes S_b unit copies and every demand a becomes D_a unit
copies (the copies of a vertex consecutive, vertices ascending).  The main
routine of Sec. 2.2, in its unbalanced form (Sec. 3.3), runs on the copies
with the round rule of the assignment oracle: each free supply copy proposes
to the lowest demand copy that is admissible (y(a) + y(b) = cbar + 1 in
units of eps) and not taken earlier in the phase, each demand copy accepts
its lowest proposer, and rounds repeat until nobody proposes.  Step II
evicts the previous partner; step III lowers the matched demand copies'
duals and raises the unmatched free supply copies' duals.  Sec. 4's
invariant then raises every free supply copy's dual to the largest dual
among the copies of its vertex.  The phases stop when at most T supply
copies are free.

The cluster oracle (ot_oracle.c) handles the copies of a vertex together
and grants a vertex's proposal as many copies as are available in one round,
evicting from the highest supplier; it is the parity target of pr_ot.  This
form chooses its maximal matchings copy by copy, so the two may differ, and
it serves to check the cluster oracle against the paper's bounds and
invariants from an independent implementation.
"""
from __future__ import annotations

import numpy as np


def ot_expanded(cb, S, D, T, phase_cap=1 << 40):
    """Run Sec. 4 on the materialised copies.

    cb: (nB, nA) integer rounded costs; S, D: copy counts per supply and
    demand vertex; T: stop when at most T supply copies are free.
    Returns a dict: counts (nB, nA) of matched copy pairs, phases, rounds,
    free (free supply copies at the stop), and the copy-level state sup, dem
    (copy -> vertex), y_sup, y_dem (duals in units of eps) and match (supply
    copy -> demand copy or -1)."""
    cb = np.asarray(cb)
    nB, nA = cb.shape
    sup = [b for b in range(nB) for _ in range(int(S[b]))]
    dem = [a for a in range(nA) for _ in range(int(D[a]))]
    nS, nD = len(sup), len(dem)
    siblings = [[i for i in range(nS) if sup[i] == b] for b in range(nB)]
    y_sup, y_dem = [1] * nS, [0] * nD
    match, owner = [-1] * nS, [-1] * nD
    phases = rounds = 0
    while True:
        free = [i for i in range(nS) if match[i] < 0]
        if len(free) <= T or phases >= phase_cap:
            break
        phases += 1
        taken = [False] * nD
        mate = {}
        resume = {i: 0 for i in free}
        active = list(free)
        while True:
            proposals = {}
            proposers = []
            for i in active:
                row = cb[sup[i]]
                p = -1
                for j in range(resume[i], nD):
                    if not taken[j] and y_dem[j] + y_sup[i] == int(row[dem[j]]) + 1:
                        p = j
                        break
                if p < 0:
                    continue
                resume[i] = p
                proposals.setdefault(p, []).append(i)
                proposers.append(i)
            if not proposals:
                break
            rounds += 1
            for j, who in proposals.items():
                taken[j] = True
                mate[min(who)] = j
            active = [i for i in proposers if i not in mate]
        for i, j in mate.items():  # step II
            if owner[j] >= 0:
                match[owner[j]] = -1
            owner[j] = i
            match[i] = j
        for j in mate.values():  # step III
            y_dem[j] -= 1
        for i in free:
            if i not in mate:
                y_sup[i] += 1
        for cs in siblings:  # Sec. 4: free copies take the largest sibling dual
            if cs:
                top = max(y_sup[i] for i in cs)
                for i in cs:
                    if match[i] < 0:
                        y_sup[i] = top
    counts = np.zeros((nB, nA), np.int64)
    for i in range(nS):
        if match[i] >= 0:
            counts[sup[i], dem[match[i]]] += 1
    return dict(counts=counts, phases=phases, rounds=rounds,
                free=sum(1 for i in range(nS) if match[i] < 0),
                sup=sup, dem=dem, y_sup=y_sup, y_dem=y_dem, match=match)


def copy_violations(r, cb) -> int:
    """Violations of the copy instance's eps-feasibility (Eqs. 2 and 3 in
    units of eps: y(a) + y(b) <= cbar + 1 on every pair, = cbar on matched
    pairs), of y(b) >= 1 >= 1 + y(a), of y(a) = 0 on free demand copies, and
    of Sec. 4's raise invariant (a free supply copy's dual is the largest
    among its vertex's copies)."""
    sup, dem, ys, yd, match = r["sup"], r["dem"], r["y_sup"], r["y_dem"], r["match"]
    nS, nD = len(sup), len(dem)
    owned = [False] * nD
    bad = 0
    for i in range(nS):
        if match[i] >= 0:
            owned[match[i]] = True
        if ys[i] < 1:
            bad += 1
        row = cb[sup[i]]
        for j in range(nD):
            s = yd[j] + ys[i]
            c = int(row[dem[j]])
            if (match[i] == j and s != c) or (match[i] != j and s > c + 1):
                bad += 1
    for j in range(nD):
        if yd[j] > 0 or (not owned[j] and yd[j] != 0):
            bad += 1
    top = {}
    for i in range(nS):
        top[sup[i]] = max(top.get(sup[i], ys[i]), ys[i])
    for i in range(nS):
        if match[i] < 0 and ys[i] < top[sup[i]]:
            bad += 1
    return bad
