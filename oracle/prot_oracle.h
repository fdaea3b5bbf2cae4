/*
 * prot_oracle.h -- the CPU oracle's own declarations (test infrastructure
 * only; independent of the CUDA library's public header).
 */
#ifndef PROT_ORACLE_H
#define PROT_ORACLE_H
#include <stdint.h>

#define OR_OK 0
#define OR_ERR_INVALID (-1)
#define OR_ERR_NO_CONVERGENCE (-4)
#define OR_ERR_NOMEM (-7)

/* mode bits of or_assign_int */
#define OR_MODE_RESUME 0      /* resume pointer per b (default)             */
#define OR_MODE_LITERAL 1     /* rescan every row from a = 0 in every round */
#define OR_MODE_CHECK 2       /* check (I1)/(I2) after every phase          */
#define OR_MODE_REVERSE 4     /* process B' in descending order             */
#define OR_MODE_SEQUENTIAL 8  /* the paper's sequential greedy (Lemma 3.4)  */
#define OR_MODE_PARALLEL 64 /* the scans of a round on all host cores (OpenMP);
                               same results                                  */
#define OR_MODE_OFFSET 32   /* step I rule with seeded start columns: in phase
                               p every free row b scans cyclically from
                               column splitmix64(p << 32 | b) mod |A|        */
#define OR_MODE_EVICT_RESUME 16 /* a row evicted in phase p starts its scan in
                                   phase p+1 after the column it lost (same
                                   results; fewer entries examined)         */
#define OR_MODE_ISRAELI_ITAI 128 /* step I by Israeli and Itai's randomized
                                    maximal matching (Sec. 3.2, parallel
                                    efficiency): every vertex points to a
                                    random neighbour, keeps one random
                                    incoming pointer, picks one of its <= 2
                                    remaining edges; edges picked at both
                                    ends join M'; repeat until maximal.
                                    Random choices are minima of seeded
                                    SplitMix64 draws (see prot_oracle.c)   */
#define OR_II_MAX_ITERS 4096     /* iterations per phase before the oracle
                                    reports no convergence                  */

typedef struct {
    int64_t phases;       /* phases executed                                  */
    int64_t rounds;       /* rounds (with at least one proposal), all phases  */
    int64_t scanned;      /* cost entries examined by the proposal scans      */
    int64_t sum_ni;       /* sum over phases of |B'|                          */
    int64_t violations;   /* invariant violations seen (OR_MODE_CHECK)        */
    int32_t free_at_stop; /* |B'| when the loop stopped                      */
    int32_t threshold;    /* T                                                */
} or_stats;

int or_quantise_f64(const double *C, int64_t ldc, int32_t nB, int32_t nA, double eps, int32_t *cb);
int or_quantise_f32(const float *C, int64_t ldc, int32_t nB, int32_t nA, double eps, int32_t *cb);
int32_t or_threshold(double eps, int32_t nB);
int64_t or_phase_cap(double eps, int32_t nB);
uint64_t or_ii_key(uint32_t step, uint32_t phase, uint32_t iter, uint32_t u, uint32_t v);
int64_t or_check_state(const int32_t *cb, int32_t nB, int32_t nA, const int32_t *match_b,
                       const int32_t *match_a, const int32_t *y_b, const int32_t *y_a);
int or_assign_int(const int32_t *cb, int32_t nB, int32_t nA, int32_t T, int32_t mode,
                  int64_t phase_cap, int32_t *match_b, int32_t *match_a, int32_t *y_b,
                  int32_t *y_a, or_stats *st, int32_t *ni_log, int64_t ni_log_cap);
void or_complete(int32_t nB, int32_t nA, int32_t *match_b, int32_t *match_a);
double or_cost_f64(const double *C, int64_t ldc, int32_t nB, const int32_t *match_b);
double or_cost_f32(const float *C, int64_t ldc, int32_t nB, const int32_t *match_b);
int or_assign_f64(const double *C, int64_t ldc, int32_t nB, int32_t nA, double eps, int32_t mode,
                  int32_t *match_b, int32_t *match_a, int32_t *y_b, int32_t *y_a, double *cost,
                  or_stats *st);
int or_assign_f32(const float *C, int64_t ldc, int32_t nB, int32_t nA, double eps, int32_t mode,
                  int32_t *match_b, int32_t *match_a, int32_t *y_b, int32_t *y_a, double *cost,
                  or_stats *st);
double or_hungarian(const double *C, int64_t ldc, int32_t nB, int32_t nA, int32_t *row_to_col);

/* optimal transport (Sec. 4), cluster form */
int or_ot_cluster_int(const int32_t *cb, int32_t nB, int32_t nA, const int32_t *S, const int32_t *D,
                      int64_t T, int32_t mode, int64_t phase_cap, int32_t *F, int32_t *f,
                      int32_t *kmin, int32_t *clo, int32_t *chi, int32_t *plan_lo,
                      int32_t *plan_hi, or_stats *st);
int64_t or_ot_check(const int32_t *cb, int32_t nB, int32_t nA, const int32_t *F, const int32_t *f,
                    const int32_t *kmin, const int32_t *clo, const int32_t *chi, const void *unused);
double or_ot_theta(int32_t nB, int32_t nA, double eps);
/* S_b = floor(theta nu_b), D_a = ceil(theta mu_a); OR_ERR_INVALID for a
 * negative or NaN mass, a mass >= 2, or a side whose floor(m 2^32) sum to
 * 1.5 * 2^32 or more (the masses must sum to 1). */
int or_ot_counts(const double *nu, const double *mu, int32_t nB, int32_t nA, double eps,
                 int32_t *S, int32_t *D);
/* mass = plan_cnt / theta, the demand trim, then the north-west corner over
 * the residuals in whole units of 2^-62; returns the FP64 cost. */
double or_ot_fixup(const double *C, int64_t ldc, int32_t nB, int32_t nA, const double *nu,
                   const double *mu, double theta, const int32_t *plan_cnt, double *mass);

/* points forms */
void or_points_cost(const float *XA, const float *XB, int32_t nA, int32_t nB, int32_t dim,
                    int32_t squared, float *C);
double or_points_match_cost(const float *XA, const float *XB, int32_t nB, int32_t dim,
                            int32_t squared, const int32_t *row_to_col);
int or_assign_points(const float *XA, const float *XB, int32_t nA, int32_t nB, int32_t dim,
                     int32_t squared, double eps, int32_t *match_b, int32_t *match_a,
                     int32_t *y_b, int32_t *y_a, double *cost, or_stats *st);
void or_sqeuclid_backward(const float *X, const float *Y, int32_t n, int32_t dim,
                          const int32_t *row_to_col, float g, float *gX, float *gY);

#endif
