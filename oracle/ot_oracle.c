/*
 * ot_oracle.c -- oracle for the optimal-transport form (Sec. 4 of Lahn,
 * Raghvendra, Zhang).  TEST INFRASTRUCTURE ONLY; shares nothing with the CUDA
 * library.
 *
 * Sec. 4: scale the masses by theta = 4n/eps, round supplies down and demands
 * up, replace each vertex by that many unit copies and run the matching
 * algorithm of Sec. 2.2 on the unbalanced copy instance (Sec. 3.3), keeping
 * the dual of every free supply copy raised to the largest dual among its
 * sibling copies (the raise rule).  This file runs that algorithm on copy
 * CLUSTERS:
 *
 *   supply b: F_b = dual of its free copies (= the largest dual of any copy
 *             of b, by the raise rule), f_b = number of free copies;
 *   demand a: its copies carry keys k = -y in {kmin_a, kmin_a + 1} (at most
 *             two clusters, Lemma 4.1): clo_a copies at kmin_a, chi_a at
 *             kmin_a + 1.  A copy is free iff its key is 0 (invariant I1).
 *
 * For a free copy of b, eps-feasibility (Eq. 2) against a's copies at kmin_a
 * forces F_b - 1 - cbar(a,b) <= kmin_a, so the only cluster of a that can be
 * admissible for b is kmin_a, and (a, b) is admissible iff
 *   cbar(b,a) + kmin_a == F_b - 1,
 * the same integer test as the assignment case with k(a) = kmin_a.
 *
 * One phase (B' = supply vertices with free copies):
 *   Step I (rounds): every b with free copies still unplaced (r_b > 0)
 *     proposes to the lowest a >= its resume column that is admissible and
 *     still has unmatched kmin-cluster copies in this phase (avail_a > 0);
 *     each a grants its lowest-index proposer g = min(r_b, avail_a) copies.
 *     Proposers resume at the same column next round.  Rounds repeat until
 *     nobody proposes; the result is a maximal matching of the copy graph.
 *   Step II: a grant taking copies of a matched cluster (kmin_a >= 1) evicts
 *     their partners, taken from a's kmin-cluster matches with the highest
 *     supply index first; each evicted copy of b'' rejoins the free copies of
 *     b'' (raised to F_b'').  The granted copies of b are matched to a at key
 *     kmin_a + 1.
 *   Step III: (a) granted copies of a move from kmin_a to kmin_a + 1; when
 *     the kmin cluster is empty the clusters shift up (kmin_a += 1);
 *     (b) every b of B' that kept unplaced free copies has F_b += 1.
 * The phases stop when at most T = floor(eps * S) supply copies are free
 * (S = total supply copies, Sec. 3.3).  With one copy per vertex this is
 * exactly the assignment routine of Sec. 2.2 (a pin in the tests).
 *
 * Plan and fix-up (the paper defers these details to LMR'19, which is not
 * available; this is the reading used): mass(b,a) = matched copies / theta.
 * Demand a that received more than mu_a gives the excess back from its
 * highest-index suppliers first; then every supply's unsent remainder is
 * routed north-west-corner style (b ascending, a ascending) into the
 * remaining demand capacity, on the remainders rounded down to whole units
 * of 2^-62 so that the rule runs in exact integer arithmetic.  cost = sum
 * mass * c, FP64, Neumaier-compensated in (b, a) ascending order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "prot_oracle.h"

/* Cluster engine on integer copy counts.  Outputs the final cluster state
 * and the matched copy counts, dense int32 [b * nA + a]: plan_lo counts the
 * copies of b matched to a's cluster at key kmin_a, plan_hi those at key
 * kmin_a + 1. */
int or_ot_cluster_int(const int32_t *cb, int32_t nB, int32_t nA, const int32_t *S,
                      const int32_t *D, int64_t T, int32_t mode, int64_t phase_cap,
                      int32_t *F, int32_t *f, int32_t *kmin, int32_t *clo, int32_t *chi,
                      int32_t *plan_lo, int32_t *plan_hi, or_stats *st)
{
    memset(st, 0, sizeof(*st));
    st->threshold = (int32_t)T;
    /* matched copy counts of the two clusters of every a, [a][b] */
    int32_t *Plo = plan_lo, *Phi = plan_hi;  /* indexed [b * nA + a] as outputs */
    int32_t *r = (int32_t *)malloc(sizeof(int32_t) * nB);
    int32_t *ptr = (int32_t *)malloc(sizeof(int32_t) * nB);
    int32_t *prop = (int32_t *)malloc(sizeof(int32_t) * nB);
    char *searching = (char *)malloc((size_t)nB);
    char *in_bp = (char *)malloc((size_t)nB);
    int32_t *avail = (int32_t *)malloc(sizeof(int32_t) * nA);
    int32_t *best = (int32_t *)malloc(sizeof(int32_t) * nA);
    int rc = OR_OK;
    if (!r || !ptr || !prop || !searching || !in_bp || !avail || !best) {
        rc = OR_ERR_NOMEM;
        goto out;
    }
    memset(Plo, 0, sizeof(int32_t) * (size_t)nB * (size_t)nA);
    memset(Phi, 0, sizeof(int32_t) * (size_t)nB * (size_t)nA);
    for (int32_t b = 0; b < nB; ++b) { F[b] = 1; f[b] = S[b]; }
    for (int32_t a = 0; a < nA; ++a) { kmin[a] = 0; clo[a] = D[a]; chi[a] = 0; best[a] = INT32_MAX; }

    for (;;) {
        int64_t nfree = 0;
        for (int32_t b = 0; b < nB; ++b) nfree += f[b];
        if (nfree <= T) { st->free_at_stop = (int32_t)nfree; break; }
        if (st->phases >= phase_cap) { st->free_at_stop = (int32_t)nfree; rc = OR_ERR_NO_CONVERGENCE; break; }
        st->phases += 1;
        for (int32_t b = 0; b < nB; ++b) {
            r[b] = f[b];
            in_bp[b] = f[b] > 0;
            searching[b] = f[b] > 0;
            ptr[b] = 0;
        }
        st->sum_ni += nfree;
        for (int32_t a = 0; a < nA; ++a) avail[a] = clo[a];

        /* Step I: rounds of proposals and grants. */
        for (;;) {
            int32_t nprop = 0;
            for (int32_t b = 0; b < nB; ++b) {
                prop[b] = -1;
                if (!searching[b]) continue;
                int32_t p = -1;
                for (int32_t a = ptr[b]; a < nA; ++a) {
                    st->scanned += 1;
                    if (avail[a] > 0 && cb[(int64_t)b * nA + a] + kmin[a] == F[b] - 1) { p = a; break; }
                }
                if (p < 0) { searching[b] = 0; continue; }
                prop[b] = p;
                ptr[b] = p;
                ++nprop;
                if (b < best[p]) best[p] = b;
            }
            if (nprop == 0) break;
            st->rounds += 1;
            /* each a grants its lowest proposer; a ascending */
            for (int32_t a = 0; a < nA; ++a) {
                const int32_t w = best[a];
                if (w == INT32_MAX) continue;
                best[a] = INT32_MAX;
                int32_t g = r[w] < avail[a] ? r[w] : avail[a];
                avail[a] -= g;
                r[w] -= g;
                /* Step II for this grant: evict from the highest supply index */
                if (kmin[a] >= 1) {
                    int32_t need = g;
                    for (int32_t b2 = nB - 1; b2 >= 0 && need > 0; --b2) {
                        int32_t *c = &Plo[(int64_t)b2 * nA + a];
                        if (*c == 0) continue;
                        int32_t t = *c < need ? *c : need;
                        *c -= t;
                        f[b2] += t;
                        need -= t;
                    }
                }
                Phi[(int64_t)w * nA + a] += g;
                f[w] -= g;
                clo[a] -= g;
                chi[a] += g;
                if (r[w] == 0) searching[w] = 0;
            }
        }
        /* Step III */
        for (int32_t b = 0; b < nB; ++b)
            if (in_bp[b] && r[b] > 0) F[b] += 1;
        for (int32_t a = 0; a < nA; ++a) {
            if (clo[a] == 0 && chi[a] > 0) {
                /* the kmin cluster is empty (its matches were all evicted or
                 * it held free copies): the clusters shift up */
                kmin[a] += 1;
                clo[a] = chi[a];
                chi[a] = 0;
                for (int32_t b = 0; b < nB; ++b) {
                    Plo[(int64_t)b * nA + a] = Phi[(int64_t)b * nA + a];
                    Phi[(int64_t)b * nA + a] = 0;
                }
            }
        }
        if (mode & OR_MODE_CHECK) st->violations += or_ot_check(cb, nB, nA, F, f, kmin, clo, chi, NULL);
    }

out:
    free(r); free(ptr); free(prop); free(searching); free(in_bp);
    free(avail); free(best);
    return rc;
}

/* Feasibility of the free supply copies against every demand cluster (the
 * part of (I2) that the cluster state determines by itself): for b with free
 * copies and every a that has copies, cbar(b,a) + kmin_a >= F_b - 1.  Also kmin >= 0 and
 * non-negative counts.  Returns the number of violations. */
int64_t or_ot_check(const int32_t *cb, int32_t nB, int32_t nA, const int32_t *F, const int32_t *f,
                    const int32_t *kmin, const int32_t *clo, const int32_t *chi, const void *unused)
{
    (void)unused;
    int64_t bad = 0;
    for (int32_t a = 0; a < nA; ++a)
        if (kmin[a] < 0 || clo[a] < 0 || chi[a] < 0) ++bad;
    for (int32_t b = 0; b < nB; ++b) {
        if (f[b] < 0 || F[b] < 1) ++bad;
        if (f[b] == 0) continue;
        for (int32_t a = 0; a < nA; ++a)   /* a column without copies constrains nothing */
            if (clo[a] + chi[a] > 0 && cb[(int64_t)b * nA + a] + kmin[a] < F[b] - 1) ++bad;
    }
    return bad;
}

/* theta = 4n/eps (n = max(nB, nA)); S_b = floor(theta nu_b), D_a = ceil(theta mu_a). */
double or_ot_theta(int32_t nB, int32_t nA, double eps)
{
    int32_t n = nB > nA ? nB : nA;
    return (4.0 * (double)n) / eps;
}

int or_ot_counts(const double *nu, const double *mu, int32_t nB, int32_t nA, double eps,
                 int32_t *S, int32_t *D)
{
    double theta = or_ot_theta(nB, nA, eps);
    for (int32_t b = 0; b < nB; ++b) {
        double v = floor(theta * nu[b]);
        if (!(nu[b] >= 0.0) || v > 2147483647.0) return OR_ERR_INVALID;
        S[b] = (int32_t)v;
    }
    for (int32_t a = 0; a < nA; ++a) {
        double v = ceil(theta * mu[a]);
        if (!(mu[a] >= 0.0) || v > 2147483647.0) return OR_ERR_INVALID;
        D[a] = (int32_t)v;
    }
    /* The masses of each side must sum to 1.  Refused: a mass of 2 or more,
     * or a side whose floor(m * 2^32) add up to 1.5 * 2^32 or more (an exact
     * integer sum, so the decision does not depend on the summation order).
     * What passes sums to below 2, which keeps the fix-up's 2^-62 units of
     * every residual and of their totals below 2^63. */
    for (int side = 0; side < 2; ++side) {
        const double *m = side ? mu : nu;
        const int32_t n = side ? nA : nB;
        uint64_t units = 0;
        for (int32_t k = 0; k < n; ++k) {
            if (!(m[k] < 2.0)) return OR_ERR_INVALID;
            units += (uint64_t)(m[k] * 0x1p32);
        }
        if (units >= 3ull << 31) return OR_ERR_INVALID;
    }
    return OR_OK;
}

static void nsum(double *s, double *comp, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *comp += (*s - t) + x;
    else *comp += (x - t) + *s;
    *s = t;
}

/* The plan from the matched counts, then the fix-up.  mass is a dense
 * nB x nA FP64 array (in/out).  Returns the FP64 cost. */
double or_ot_fixup(const double *C, int64_t ldc, int32_t nB, int32_t nA, const double *nu,
                   const double *mu, double theta, const int32_t *plan_cnt, double *mass)
{
    for (int32_t b = 0; b < nB; ++b)
        for (int32_t a = 0; a < nA; ++a)
            mass[(int64_t)b * nA + a] = (double)plan_cnt[(int64_t)b * nA + a] / theta;
    double *q = (double *)malloc(sizeof(double) * nA);
    double *rres = (double *)malloc(sizeof(double) * nB);
    /* demand side: give back any excess over mu_a, highest b first */
    for (int32_t a = 0; a < nA; ++a) {
        double recv = 0.0;
        for (int32_t b = 0; b < nB; ++b) recv += mass[(int64_t)b * nA + a];
        double excess = recv - mu[a];
        for (int32_t b = nB - 1; b >= 0 && excess > 0.0; --b) {
            double *m = &mass[(int64_t)b * nA + a];
            if (*m <= 0.0) continue;
            double t = *m < excess ? *m : excess;
            *m -= t;
            excess -= t;
        }
        double r2 = 0.0;
        for (int32_t b = 0; b < nB; ++b) r2 += mass[(int64_t)b * nA + a];
        q[a] = mu[a] - r2;
        if (q[a] < 0.0) q[a] = 0.0;
    }
    for (int32_t b = 0; b < nB; ++b) {
        double sent = 0.0;
        for (int32_t a = 0; a < nA; ++a) sent += mass[(int64_t)b * nA + a];
        rres[b] = nu[b] - sent;
        if (rres[b] < 0.0) rres[b] = 0.0;
    }
    /* North-west corner over the residuals, in exact integer units of 2^-62:
     * each residual is first rounded down to a whole number of units (the
     * product by 2^62 is exact; it loses less than 2^-62 per vertex), the
     * rule then runs on integers, and each allocation becomes t * 2^-62 in
     * FP64 (one rounding, to nearest). */
    uint64_t *ru = (uint64_t *)malloc(sizeof(uint64_t) * nB);
    uint64_t *qu = (uint64_t *)malloc(sizeof(uint64_t) * nA);
    for (int32_t b = 0; b < nB; ++b) ru[b] = rres[b] > 0.0 ? (uint64_t)(rres[b] * 0x1p62) : 0;
    for (int32_t a = 0; a < nA; ++a) qu[a] = q[a] > 0.0 ? (uint64_t)(q[a] * 0x1p62) : 0;
    int32_t i = 0, j = 0;
    while (i < nB && j < nA) {
        if (ru[i] == 0) { ++i; continue; }
        if (qu[j] == 0) { ++j; continue; }
        uint64_t t = ru[i] < qu[j] ? ru[i] : qu[j];
        mass[(int64_t)i * nA + j] += (double)t * 0x1p-62;
        ru[i] -= t;
        qu[j] -= t;
    }
    free(ru);
    free(qu);
    double s = 0.0, comp = 0.0;
    for (int32_t b = 0; b < nB; ++b)
        for (int32_t a = 0; a < nA; ++a) {
            double m = mass[(int64_t)b * nA + a];
            if (m != 0.0) nsum(&s, &comp, m * C[(int64_t)b * ldc + a]);
        }
    free(q);
    free(rres);
    return s + comp;
}
