/*
 * prot_oracle.c -- plain, slow CPU oracle for the push-relabel additive
 * approximation of Lahn, Raghvendra and Zhang, "A Push-Relabel Based Additive
 * Approximation for Optimal Transport" (arXiv 2203.03732).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package's smoke entry and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library: it is written from the paper alone, as nested loops over
 * plain arrays, in the order the paper states its steps.
 *
 * Units: every dual weight and rounded cost is kept as an integer multiple of
 * eps (Sec. 2.1 says all duals stay integer multiples of eps), so
 *   cb(b,a) = floor(c(b,a) / eps), exact quotient (Eq. 1, divided by eps)
 *   admissible(a,b)  <=>  y(a) + y(b) == cb + 1   (slack 0, Sec. 2.1 / Eq. 2)
 *   matched edge     <=>  y(a) + y(b) == cb       (Eq. 3)
 * Rows are the vertices of B (the supply side whose free vertices form B'),
 * columns the vertices of A.
 *
 * Pinned choices where the paper leaves a free hand (see the design notes):
 *   - Step I's maximal matching uses the round rule: every still-active free
 *     b proposes to the lowest-index admissible a that was not taken in an
 *     earlier round of this phase; every a accepts its lowest-index proposer;
 *     rounds repeat until nobody proposes.
 *   - Completion matches the k-th free b (ascending) with the k-th free a
 *     (ascending); duals are left unchanged.
 *   - The stopping threshold is T = floor(eps * |B|) computed in FP64.
 *
 * Parity pins (all in the CPU test suite): brute force over permutations for
 * n <= 8, an exact Hungarian solver cross-checked against scipy, the
 * invariants (I1)/(I2) after every phase, Lemma 2.1, Lemma 3.1's additive
 * bound and its dual certificate, Lemma 3.2's dual magnitude bound, the exact
 * per-phase growth of Lemma 3.3, closed-form special cases (constant costs,
 * zero diagonal, zero permutation), literal-rescan vs resume-pointer
 * equivalence, and independence from the order in which B' is processed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#include "prot_oracle.h"

/* ------------------------------------------------------------------------ */
/* Eq. (1): rounding of costs to integer multiples of eps.                   */
/* ------------------------------------------------------------------------ */

/* Eq. (1) in eps units: cb = floor(c / eps) of the EXACT real quotient of
 * the two given FP64 numbers, i.e. the largest integer k with k * eps <= c.
 * The comparison k * eps <= c is decided exactly: fma(-k, eps, c) forms
 * c - k*eps exactly and rounds once, which keeps its sign (no underflow can
 * occur for k >= 1 since eps > 3e-5).  A rounded division gives a start value
 * within one of the answer.  Costs must be finite and in [0, 1] (Sec. 1
 * assumes the costs are scaled so that the largest is 1). */
static int32_t exact_floor_div(double c, double eps)
{
    int32_t k = (int32_t)floor(c / eps);
    while (k > 0 && fma(-(double)k, eps, c) < 0.0) --k;
    while (fma(-(double)(k + 1), eps, c) >= 0.0) ++k;
    return k;
}

/* Returns 0, or -1 at the first invalid cost. */
int or_quantise_f64(const double *C, int64_t ldc, int32_t nB, int32_t nA,
                    double eps, int32_t *cb)
{
    for (int32_t b = 0; b < nB; ++b) {
        for (int32_t a = 0; a < nA; ++a) {
            double c = C[(int64_t)b * ldc + a];
            if (!(c >= 0.0 && c <= 1.0)) return -1;
            cb[(int64_t)b * nA + a] = exact_floor_div(c, eps);
        }
    }
    return 0;
}

/* Same for FP32 costs: the float is first widened (exactly) to double. */
int or_quantise_f32(const float *C, int64_t ldc, int32_t nB, int32_t nA,
                    double eps, int32_t *cb)
{
    for (int32_t b = 0; b < nB; ++b) {
        for (int32_t a = 0; a < nA; ++a) {
            double c = (double)C[(int64_t)b * ldc + a];
            if (!(c >= 0.0 && c <= 1.0)) return -1;
            cb[(int64_t)b * nA + a] = exact_floor_div(c, eps);
        }
    }
    return 0;
}

/* Termination threshold of Sec. 2.2 (|B'| <= eps n), for the unbalanced case
 * with |B| <= |A| (Sec. 3.3, Lemma 3.5): T = floor(eps * |B|). */
int32_t or_threshold(double eps, int32_t nB)
{
    return (int32_t)floor(eps * (double)nB);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2: the phase loop.                                                 */
/* ------------------------------------------------------------------------ */

static int admissible(const int32_t *cb, int32_t nA, const int32_t *y_b,
                      const int32_t *y_a, int32_t b, int32_t a)
{
    return y_a[a] + y_b[b] == cb[(int64_t)b * nA + a] + 1;
}

/* Invariants (I1), (I2) and the matching's consistency.  Returns the number
 * of violations found (0 when the state is eps-feasible). */
int64_t or_check_state(const int32_t *cb, int32_t nB, int32_t nA,
                       const int32_t *match_b, const int32_t *match_a,
                       const int32_t *y_b, const int32_t *y_a)
{
    int64_t bad = 0;
    for (int32_t b = 0; b < nB; ++b) {
        int32_t a = match_b[b];
        if (a >= 0 && (a >= nA || match_a[a] != b)) ++bad;
        if (y_b[b] < 0) ++bad;                     /* (I1): y(b) >= 0 */
    }
    for (int32_t a = 0; a < nA; ++a) {
        int32_t b = match_a[a];
        if (b >= 0 && (b >= nB || match_b[b] != a)) ++bad;
        if (y_a[a] > 0) ++bad;                     /* (I1): y(a) <= 0 */
        if (b < 0 && y_a[a] != 0) ++bad;           /* (I1): free a has 0 */
    }
    for (int32_t b = 0; b < nB; ++b) {
        for (int32_t a = 0; a < nA; ++a) {
            int32_t s = y_a[a] + y_b[b];
            int32_t c = cb[(int64_t)b * nA + a];
            if (match_b[b] == a) {
                if (s != c) ++bad;                 /* Eq. (3) */
            } else {
                if (s > c + 1) ++bad;              /* Eq. (2) */
            }
        }
    }
    return bad;
}

/* SplitMix64's output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): the seeded start columns
 * of OR_MODE_OFFSET are splitmix64(phase << 32 | b) mod |A|. */
static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

/* ------------------------------------------------------------------------ */
/* Step I by Israeli and Itai's randomized maximal matching (A. Israeli and  */
/* A. Itai, "A fast and simple randomized parallel algorithm for maximal     */
/* matching", IPL 22, 1986), which Sec. 3.2 names for the O(log n) parallel  */
/* bound of a phase.  One iteration on the admissible graph of the phase's   */
/* free rows and untaken columns:                                            */
/*   1. every vertex with an edge points to one neighbour, chosen uniformly; */
/*   2. every vertex pointed at keeps one of the pointers, chosen uniformly; */
/*   3. the kept pointers leave every vertex at most two edges; it picks one */
/*      of them, uniformly; an edge picked by both its ends joins M'.        */
/* Matched vertices, and rows with no edge left, leave; the iterations go on */
/* while some row has an edge, so M' ends maximal.                           */
/*                                                                           */
/* A uniform choice among candidates is the candidate with the least key,    */
/* key = (draw >> 24) << 24 | candidate index: 40 random bits, then the      */
/* index (which also settles ties); a choice between two edges in step 3     */
/* takes the low bit of a draw.  Draws are three SplitMix64 rounds (Steele,  */
/* Lea and Flood 2014) over (step, phase, iteration), then the vertex, then  */
/* the other end; vertex ids are b for row b and 2^24 + a for column a.      */
/* ------------------------------------------------------------------------ */
#define II_COL (1u << 24)

static uint64_t ii_draw(uint32_t step, uint32_t phase, uint32_t iter, uint32_t u, uint32_t v)
{
    uint64_t x = splitmix64(((uint64_t)step << 56) ^ ((uint64_t)phase << 28) ^ (uint64_t)iter);
    x = splitmix64(x ^ (uint64_t)u);
    return splitmix64(x ^ (uint64_t)v);
}

/* Key of candidate v (an index below 2^24) for vertex u. */
uint64_t or_ii_key(uint32_t step, uint32_t phase, uint32_t iter, uint32_t u, uint32_t v)
{
    return ((ii_draw(step, phase, iter, u, v) >> 24) << 24) | (uint64_t)(v & 0xFFFFFFu);
}

/* One phase's step I by the randomized rule: mate[b] for b in F (-1: none),
 * taken[a] = 1 for the columns of M'.  Returns the iterations with an edge,
 * or -1 when OR_II_MAX_ITERS iterations did not make M' maximal. */
static int64_t israeli_itai_phase(const int32_t *cb, int32_t nB, int32_t nA, const int32_t *y_b,
                                  const int32_t *y_a, const int32_t *F, int32_t nf, uint32_t phase,
                                  int32_t *mate, int32_t *taken, int64_t *scanned)
{
    const uint64_t NONE = UINT64_MAX;
    int32_t *act = (int32_t *)malloc(sizeof(int32_t) * (size_t)nB);
    int32_t *rp = (int32_t *)malloc(sizeof(int32_t) * (size_t)nB);   /* step 1, rows    */
    int32_t *rc = (int32_t *)malloc(sizeof(int32_t) * (size_t)nB);   /* step 3, rows    */
    int32_t *cc = (int32_t *)malloc(sizeof(int32_t) * (size_t)nA);   /* step 3, columns */
    uint64_t *cp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nA);   /* step 1, columns */
    uint64_t *cin = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nA);  /* step 2, columns */
    uint64_t *rin = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nB);  /* step 2, rows    */
    int64_t rounds = 0;
    for (int32_t b = 0; b < nB; ++b) act[b] = 0;
    for (int32_t i = 0; i < nf; ++i) act[F[i]] = 1;
    for (uint32_t it = 1;; ++it) {
        if (it > OR_II_MAX_ITERS) { rounds = -1; break; }
        /* step 1: rows and columns point to a neighbour */
        int32_t any = 0;
        for (int32_t a = 0; a < nA; ++a) cp[a] = NONE;
        for (int32_t b = 0; b < nB; ++b) {
            rp[b] = -1;
            if (!act[b]) continue;
            uint64_t best = NONE;
            for (int32_t a = 0; a < nA; ++a) {
                *scanned += 1;
                if (taken[a] || y_a[a] + y_b[b] != cb[(int64_t)b * nA + a] + 1) continue;
                uint64_t kr = or_ii_key(1, phase, it, (uint32_t)b, (uint32_t)a);
                if (kr < best) { best = kr; rp[b] = a; }
                uint64_t kc = or_ii_key(1, phase, it, II_COL + (uint32_t)a, (uint32_t)b);
                if (kc < cp[a]) cp[a] = kc;
            }
            if (rp[b] < 0) act[b] = 0;   /* no edge left: relabelled at the phase end */
            else any = 1;
        }
        if (!any) break;
        rounds += 1;
        /* step 2: keep one incoming pointer */
        for (int32_t a = 0; a < nA; ++a) cin[a] = NONE;
        for (int32_t b = 0; b < nB; ++b) rin[b] = NONE;
        for (int32_t b = 0; b < nB; ++b) {
            if (rp[b] < 0) continue;
            int32_t a = rp[b];
            uint64_t k = or_ii_key(2, phase, it, II_COL + (uint32_t)a, (uint32_t)b);
            if (k < cin[a]) cin[a] = k;
        }
        for (int32_t a = 0; a < nA; ++a) {
            if (cp[a] == NONE) continue;
            int32_t b = (int32_t)(cp[a] & 0xFFFFFFu);
            uint64_t k = or_ii_key(2, phase, it, (uint32_t)b, (uint32_t)a);
            if (k < rin[b]) rin[b] = k;
        }
        /* step 3: every vertex picks one of its remaining edges */
        for (int32_t b = 0; b < nB; ++b) {
            rc[b] = -1;
            if (!act[b]) continue;
            int32_t out = (rp[b] >= 0 && cin[rp[b]] != NONE && (int32_t)(cin[rp[b]] & 0xFFFFFFu) == b) ? rp[b] : -1;
            int32_t in = rin[b] != NONE ? (int32_t)(rin[b] & 0xFFFFFFu) : -1;
            if (out >= 0 && in >= 0)
                rc[b] = (ii_draw(3, phase, it, (uint32_t)b, 0) & 1) ? in : out;
            else
                rc[b] = out >= 0 ? out : in;
        }
        for (int32_t a = 0; a < nA; ++a) {
            cc[a] = -1;
            if (taken[a]) continue;
            int32_t out = -1;
            if (cp[a] != NONE) {
                int32_t b = (int32_t)(cp[a] & 0xFFFFFFu);
                if (rin[b] != NONE && (int32_t)(rin[b] & 0xFFFFFFu) == a) out = b;
            }
            int32_t in = cin[a] != NONE ? (int32_t)(cin[a] & 0xFFFFFFu) : -1;
            if (out >= 0 && in >= 0)
                cc[a] = (ii_draw(3, phase, it, II_COL + (uint32_t)a, 0) & 1) ? in : out;
            else
                cc[a] = out >= 0 ? out : in;
        }
        /* edges picked at both ends join M' */
        for (int32_t b = 0; b < nB; ++b) {
            int32_t a = rc[b];
            if (a >= 0 && cc[a] == b) { mate[b] = a; taken[a] = 1; act[b] = 0; }
        }
    }
    free(act); free(rp); free(rc); free(cc); free(cp); free(cin); free(rin);
    return rounds;
}

/*
 * One run of the main routine of Sec. 2.2 on integer costs cb (row-major,
 * nB x nA, nB <= nA).  Outputs the matching before completion and both dual
 * vectors.  mode is a bit set of OR_MODE_*.
 *
 * Returns OR_OK, OR_ERR_NO_CONVERGENCE if phase_cap phases ran without
 * reaching the threshold, OR_ERR_INVALID for bad sizes, OR_ERR_NOMEM.
 */
int or_assign_int(const int32_t *cb, int32_t nB, int32_t nA, int32_t T,
                  int32_t mode, int64_t phase_cap,
                  int32_t *match_b, int32_t *match_a,
                  int32_t *y_b, int32_t *y_a, or_stats *st,
                  int32_t *ni_log, int64_t ni_log_cap)
{
    if (nB < 1 || nA < nB || T < 0) return OR_ERR_INVALID;
    int32_t *F = (int32_t *)malloc(sizeof(int32_t) * nB);      /* B' */
    int32_t *act = (int32_t *)malloc(sizeof(int32_t) * nB);    /* active */
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * nB);
    int32_t *mate = (int32_t *)malloc(sizeof(int32_t) * nB);   /* M' */
    int32_t *ptr = (int32_t *)malloc(sizeof(int32_t) * nB);
    int32_t *prop = (int32_t *)malloc(sizeof(int32_t) * nB);
    int32_t *taken = (int32_t *)malloc(sizeof(int32_t) * nA);  /* round */
    int32_t *best = (int32_t *)malloc(sizeof(int32_t) * nA);
    int32_t *mround = (int32_t *)malloc(sizeof(int32_t) * nB);
    int32_t *resume = (int32_t *)calloc((size_t)nB, sizeof(int32_t));
    int32_t *covered = (int32_t *)calloc((size_t)nB, sizeof(int32_t));  /* OR_MODE_OFFSET */
    if (!F || !act || !nxt || !mate || !ptr || !prop || !taken || !best || !mround || !resume ||
        !covered) {
        free(F); free(act); free(nxt); free(mate); free(ptr); free(prop);
        free(taken); free(best); free(mround); free(resume); free(covered);
        return OR_ERR_NOMEM;
    }
    memset(st, 0, sizeof(*st));
    st->threshold = T;

    /* Initialisation (Sec. 2.2): y(b) = eps, y(a) = 0, M empty. */
    for (int32_t b = 0; b < nB; ++b) { y_b[b] = 1; match_b[b] = -1; }
    for (int32_t a = 0; a < nA; ++a) { y_a[a] = 0; match_a[a] = -1; best[a] = INT32_MAX; }

    int rc = OR_OK;
    for (;;) {
        /* B' = free vertices of B. */
        int32_t nf = 0;
        for (int32_t b = 0; b < nB; ++b)
            if (match_b[b] < 0) F[nf++] = b;
        if (nf <= T) { st->free_at_stop = nf; break; }
        if (st->phases >= phase_cap) { st->free_at_stop = nf; rc = OR_ERR_NO_CONVERGENCE; break; }
        if (ni_log && st->phases < ni_log_cap) ni_log[st->phases] = nf;
        st->phases += 1;
        st->sum_ni += nf;

        /* Step (I): maximal matching M' in G'(A' u B', E') by rounds. */
        for (int32_t a = 0; a < nA; ++a) taken[a] = 0;
        for (int32_t i = 0; i < nf; ++i) {
            int32_t b = F[i];
            mate[b] = -1; ptr[b] = 0; mround[b] = 0;
            /* OR_MODE_EVICT_RESUME: resume[b] = r > 0 means b was evicted
             * from column r - 1 in the previous phase.  Every column below r
             * is then inadmissible for b for good.  Column r - 1 was matched
             * to b (Eq. 3: y(a) + y(b) = cb) and y(a) dropped when it was
             * won again.  The scan that gave b column r - 1 passed the
             * columns below it as inadmissible or taken in an earlier round
             * (taken columns dropped at that phase's end).  Since then y(b)
             * has not moved (b was matched), y(a) only drops, and dual
             * feasibility (Eq. 2) never lets y(a) + y(b) exceed cb + 1, so
             * none of them returns to equality.  Starting at r gives the
             * same proposals. */
            if (mode & OR_MODE_EVICT_RESUME) ptr[b] = resume[b];
            resume[b] = 0;
            if (mode & OR_MODE_OFFSET) {
                ptr[b] = (int32_t)(splitmix64(((uint64_t)st->phases << 32) | (uint32_t)b) % (uint64_t)nA);
                covered[b] = 0;
            }
        }
        int32_t nact = nf;
        for (int32_t i = 0; i < nf; ++i) act[i] = F[i];
        if (mode & OR_MODE_REVERSE) {
            for (int32_t i = 0; i < nact / 2; ++i) {
                int32_t t = act[i]; act[i] = act[nact - 1 - i]; act[nact - 1 - i] = t;
            }
        }

        if (mode & OR_MODE_ISRAELI_ITAI) {
            int64_t r = israeli_itai_phase(cb, nB, nA, y_b, y_a, F, nf, (uint32_t)st->phases, mate, taken,
                                           &st->scanned);
            if (r < 0) { rc = OR_ERR_NO_CONVERGENCE; break; }
            st->rounds += r;
        } else if (mode & OR_MODE_SEQUENTIAL) {
            /* The paper's sequential greedy (Lemma 3.4): process B' in
             * ascending order, give each b its first admissible a that is not
             * yet matched in M'.  A different, equally valid maximal M'. */
            for (int32_t i = 0; i < nf; ++i) {
                int32_t b = F[i];
                for (int32_t a = 0; a < nA; ++a) {
                    st->scanned += 1;
                    if (!taken[a] && admissible(cb, nA, y_b, y_a, b, a)) {
                        taken[a] = 1; mate[b] = a; break;
                    }
                }
            }
            st->rounds += 1;
        } else {
            int32_t r = 0;
            for (;;) {
                ++r;
                /* Proposals of round r, all made against the taken[] state
                 * left by rounds 1..r-1. */
                /* The scans of a round read only the taken[] state and duals
                 * fixed for the round and write per-row state, so they may
                 * run in any order or at once (OR_MODE_PARALLEL: OpenMP over
                 * the active rows, for timing on all host cores); the
                 * lowest proposer of each column is taken afterwards. */
                int64_t scanned = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : scanned) if (mode & OR_MODE_PARALLEL)
                for (int32_t i = 0; i < nact; ++i) {
                    int32_t b = act[i];
                    int32_t start = (mode & OR_MODE_LITERAL) ? 0 : ptr[b];
                    int32_t p = -1;
                    if (mode & OR_MODE_OFFSET) {
                        /* cyclic scan from the row's start column; a loser
                         * goes on after the column it lost, until every
                         * column has been seen once in this phase */
                        while (covered[b] < nA) {
                            int32_t a = ptr[b];
                            ptr[b] = (a + 1 == nA) ? 0 : a + 1;
                            covered[b] += 1;
                            scanned += 1;
                            if (taken[a] == 0 && admissible(cb, nA, y_b, y_a, b, a)) { p = a; break; }
                        }
                    } else
                    for (int32_t a = start; a < nA; ++a) {
                        scanned += 1;
                        if (taken[a] == 0 && admissible(cb, nA, y_b, y_a, b, a)) { p = a; break; }
                    }
                    prop[b] = p;
                    if (p < 0) ptr[b] = nA;
                }
                st->scanned += scanned;
                int32_t nprop = 0;
                for (int32_t i = 0; i < nact; ++i) {
                    int32_t b = act[i];
                    int32_t p = prop[b];
                    if (p >= 0) {
                        ++nprop;
                        if (b < best[p]) best[p] = b;
                    }
                }
                if (nprop == 0) break;
                st->rounds += 1;
                /* Acceptance: each a takes its lowest-index proposer. */
                int32_t nn = 0;
                for (int32_t i = 0; i < nact; ++i) {
                    int32_t b = act[i];
                    int32_t p = prop[b];
                    if (p < 0) continue;              /* b leaves: no edge */
                    if (best[p] == b) {
                        mate[b] = p; mround[b] = r;
                    } else {
                        if (!(mode & OR_MODE_OFFSET)) ptr[b] = p + 1;  /* resume after p */
                        nxt[nn++] = b;
                    }
                }
                for (int32_t i = 0; i < nact; ++i) {
                    int32_t b = act[i];
                    int32_t p = prop[b];
                    if (p >= 0) { taken[p] = r; best[p] = INT32_MAX; }
                }
                nact = nn;
                for (int32_t i = 0; i < nn; ++i) act[i] = nxt[i];
                if (nact == 0) break;
            }
        }

        /* Step (II): add M' to M, delete M'' (the old edges of re-matched a).
         * Lemma 2.1: the result is a matching and no matched a becomes free. */
        if (mode & OR_MODE_CHECK)
            for (int32_t a = 0; a < nA; ++a) best[a] = match_a[a] >= 0 ? 1 : 0;
        for (int32_t i = 0; i < nf; ++i) {
            int32_t b = F[i];
            int32_t a = mate[b];
            if (a < 0) continue;
            int32_t old = match_a[a];
            if (old >= 0) { match_b[old] = -1; resume[old] = a + 1; }
            match_a[a] = b;
            match_b[b] = a;
        }
        /* Step (III): (a) y(a) -= eps for a matched in M';
         *             (b) y(b) += eps for b in B' free with respect to M'. */
        for (int32_t i = 0; i < nf; ++i) {
            int32_t b = F[i];
            if (mate[b] >= 0) y_a[mate[b]] -= 1;
            else y_b[b] += 1;
        }
        if (mode & OR_MODE_CHECK) {
            for (int32_t a = 0; a < nA; ++a) {
                if (best[a] == 1 && match_a[a] < 0) ++st->violations;   /* Lemma 2.1 */
                best[a] = INT32_MAX;
            }
            st->violations += or_check_state(cb, nB, nA, match_b, match_a, y_b, y_a);
        }
    }

    free(F); free(act); free(nxt); free(mate); free(ptr); free(prop);
    free(taken); free(best); free(mround); free(resume); free(covered);
    return rc;
}

/* Completion (Sec. 2.1, last paragraph): the remaining free vertices are
 * matched arbitrarily; pinned here as the k-th free b with the k-th free a. */
void or_complete(int32_t nB, int32_t nA, int32_t *match_b, int32_t *match_a)
{
    int32_t a = 0;
    for (int32_t b = 0; b < nB; ++b) {
        if (match_b[b] >= 0) continue;
        while (a < nA && match_a[a] >= 0) ++a;
        if (a >= nA) return;                       /* cannot happen: nB <= nA */
        match_b[b] = a;
        match_a[a] = b;
    }
}

/* c(M) = sum over the matching of the ORIGINAL costs (Sec. 1), as an FP64
 * Neumaier-compensated sum in ascending b. */
static void neumaier_add(double *s, double *comp, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *comp += (*s - t) + x;
    else *comp += (x - t) + *s;
    *s = t;
}

double or_cost_f64(const double *C, int64_t ldc, int32_t nB, const int32_t *match_b)
{
    double s = 0.0, comp = 0.0;
    for (int32_t b = 0; b < nB; ++b)
        neumaier_add(&s, &comp, C[(int64_t)b * ldc + match_b[b]]);
    return s + comp;
}

double or_cost_f32(const float *C, int64_t ldc, int32_t nB, const int32_t *match_b)
{
    double s = 0.0, comp = 0.0;
    for (int32_t b = 0; b < nB; ++b)
        neumaier_add(&s, &comp, (double)C[(int64_t)b * ldc + match_b[b]]);
    return s + comp;
}

/* Whole solve on FP64 costs: quantise, main routine, completion, cost. */
int or_assign_f64(const double *C, int64_t ldc, int32_t nB, int32_t nA, double eps,
                  int32_t mode, int32_t *match_b, int32_t *match_a,
                  int32_t *y_b, int32_t *y_a, double *cost, or_stats *st)
{
    if (nB < 1 || nA < nB || !(eps > 0.0 && eps < 1.0)) return OR_ERR_INVALID;
    if (floor(1.0 / eps) > 32766.0) return OR_ERR_INVALID;
    int32_t *cb = (int32_t *)malloc(sizeof(int32_t) * (size_t)nB * (size_t)nA);
    if (!cb) return OR_ERR_NOMEM;
    if (or_quantise_f64(C, ldc, nB, nA, eps, cb) != 0) { free(cb); return OR_ERR_INVALID; }
    int32_t T = or_threshold(eps, nB);
    int rc = or_assign_int(cb, nB, nA, T, mode, or_phase_cap(eps, nB), match_b, match_a,
                           y_b, y_a, st, NULL, 0);
    free(cb);
    if (rc != OR_OK) return rc;
    or_complete(nB, nA, match_b, match_a);
    *cost = or_cost_f64(C, ldc, nB, match_b);
    return OR_OK;
}

int or_assign_f32(const float *C, int64_t ldc, int32_t nB, int32_t nA, double eps,
                  int32_t mode, int32_t *match_b, int32_t *match_a,
                  int32_t *y_b, int32_t *y_a, double *cost, or_stats *st)
{
    if (nB < 1 || nA < nB || !(eps > 0.0 && eps < 1.0)) return OR_ERR_INVALID;
    if (floor(1.0 / eps) > 32766.0) return OR_ERR_INVALID;
    int32_t *cb = (int32_t *)malloc(sizeof(int32_t) * (size_t)nB * (size_t)nA);
    if (!cb) return OR_ERR_NOMEM;
    if (or_quantise_f32(C, ldc, nB, nA, eps, cb) != 0) { free(cb); return OR_ERR_INVALID; }
    int32_t T = or_threshold(eps, nB);
    int rc = or_assign_int(cb, nB, nA, T, mode, or_phase_cap(eps, nB), match_b, match_a,
                           y_b, y_a, st, NULL, 0);
    free(cb);
    if (rc != OR_OK) return rc;
    or_complete(nB, nA, match_b, match_a);
    *cost = or_cost_f32(C, ldc, nB, match_b);
    return OR_OK;
}

/* A phase cap that valid input never reaches.  Each phase raises the total
 * dual magnitude S = sum y(b) - sum y(a) by exactly |B'| > T (Lemma 3.3's
 * argument, made exact in integer units), S starts at |B| and, by Lemma 3.2
 * (|y| <= floor(1/eps) + 2 in eps units), ends at most 2|B|(floor(1/eps)+2).
 * Hence phases <= |B|(2 floor(1/eps) + 3) / (T + 1). */
int64_t or_phase_cap(double eps, int32_t nB)
{
    int64_t K = (int64_t)floor(1.0 / eps);
    int64_t T = or_threshold(eps, nB);
    return ((int64_t)nB * (2 * K + 3)) / (T + 1) + 1;
}

/* ------------------------------------------------------------------------ */
/* Exact solver for the pins: the textbook shortest-augmenting-path          */
/* Hungarian method with vertex potentials, O(nB^2 nA), for nB <= nA.        */
/* ------------------------------------------------------------------------ */
double or_hungarian(const double *C, int64_t ldc, int32_t nB, int32_t nA, int32_t *row_to_col)
{
    /* 1-based arrays; index 0 is the virtual root column. */
    double *u = (double *)calloc((size_t)nB + 1, sizeof(double));
    double *v = (double *)calloc((size_t)nA + 1, sizeof(double));
    double *minv = (double *)malloc(sizeof(double) * ((size_t)nA + 1));
    int32_t *p = (int32_t *)calloc((size_t)nA + 1, sizeof(int32_t));   /* row matched to column */
    int32_t *way = (int32_t *)calloc((size_t)nA + 1, sizeof(int32_t));
    char *used = (char *)malloc((size_t)nA + 1);
    for (int32_t i = 1; i <= nB; ++i) {
        p[0] = i;
        int32_t j0 = 0;
        for (int32_t j = 0; j <= nA; ++j) { minv[j] = DBL_MAX; used[j] = 0; }
        do {
            used[j0] = 1;
            int32_t i0 = p[j0], j1 = 0;
            double delta = DBL_MAX;
            for (int32_t j = 1; j <= nA; ++j) {
                if (used[j]) continue;
                double cur = C[(int64_t)(i0 - 1) * ldc + (j - 1)] - u[i0] - v[j];
                if (cur < minv[j]) { minv[j] = cur; way[j] = j0; }
                if (minv[j] < delta) { delta = minv[j]; j1 = j; }
            }
            for (int32_t j = 0; j <= nA; ++j) {
                if (used[j]) { u[p[j]] += delta; v[j] -= delta; }
                else minv[j] -= delta;
            }
            j0 = j1;
        } while (p[j0] != 0);
        do {
            int32_t j1 = way[j0];
            p[j0] = p[j1];
            j0 = j1;
        } while (j0);
    }
    for (int32_t j = 1; j <= nA; ++j)
        if (p[j] != 0) row_to_col[p[j] - 1] = j - 1;
    double s = 0.0, comp = 0.0;
    for (int32_t b = 0; b < nB; ++b)
        neumaier_add(&s, &comp, C[(int64_t)b * ldc + row_to_col[b]]);
    free(u); free(v); free(minv); free(p); free(way); free(used);
    return s + comp;
}
