/*
 * prot.h -- C ABI of the GB300 push-relabel additive-approximation solver.
 *
 * Method: Lahn, Raghvendra, Zhang, "A Push-Relabel Based Additive
 * Approximation for Optimal Transport" (arXiv 2203.03732).
 *
 * Conventions shared by every entry point
 *   - Pointers are DEVICE pointers unless a comment says "host".  The caller
 *     owns every buffer; the library never allocates device memory.  Scratch
 *     space is the caller's workspace `ws` of at least the bytes returned by
 *     the matching *_workspace() query, 256-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it in order; nothing else is touched,
 *     except by pr_assign_staged, whose host-to-device copies run on a copy
 *     stream of the library's own (ordered after the work already on
 *     `stream`; see there).
 *   - Rows are the supply side B (the side whose free vertices propose, the
 *     set B' of Sec. 2.2); columns are the demand side A.  Costs are row-major
 *     with leading dimension `ldc` (elements).  The paper assumes the costs are
 *     scaled so the largest is 1 (Sec. 1): every cost must be finite and in
 *     [0, 1]; out-of-range costs make the call fail with PR_ERR_INVALID.
 *   - Dual weights are returned as integers in units of eps (the paper keeps
 *     every dual an integer multiple of eps, Sec. 2.2): y(v) = eps * y_int.
 *   - Errors are returned as a status, never thrown.  A host-checked argument
 *     error returns before anything is enqueued.  Errors found on the device
 *     (cost out of range, barrier time-out, phase cap) are reported when the
 *     call synchronises, which it does iff `stats` is non-NULL; otherwise
 *     pr_ws_status() reads them later.  Outputs are unspecified on error.
 *   - pr_last_error() returns a thread-local message for the last failure.
 */
#ifndef PROT_H
#define PROT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PR_OK = 0,
    PR_ERR_INVALID = -1,         /* bad argument or cost outside [0,1]        */
    PR_ERR_CUDA = -2,            /* a CUDA runtime call failed                */
    PR_ERR_TIMEOUT = -3,         /* a device-side wait exceeded its budget    */
    PR_ERR_NO_CONVERGENCE = -4,  /* phase cap reached (never for valid input) */
    PR_ERR_WORKSPACE = -5,       /* workspace NULL, misaligned or too small   */
    PR_ERR_CAPACITY = -6,        /* an output buffer is too small             */
    PR_ERR_INTERNAL = -7         /* a device-side consistency check failed    */
} pr_status;

typedef enum { PR_F32 = 0, PR_F64 = 1 } pr_dtype;

/* Counters of one solve (host struct). */
typedef struct {
    int64_t phases;        /* phases of Sec. 2.2 executed                       */
    int64_t rounds;        /* rounds of step (I) in which a vertex proposed     */
    int64_t bytes_scanned; /* bytes of rounded-cost rows the row scans loaded   */
    int64_t rows_scanned;  /* row scans started (one per free vertex per round) */
    int32_t free_at_stop;  /* |B'| when the loop stopped (<= threshold)         */
    int32_t threshold;     /* T = floor(eps * n_rows)                           */
    int32_t loop_ctas;     /* CTAs that ran the phase loop (0: not applicable)  */
    int32_t loop_cluster;  /* 1: they formed one thread-block cluster; 0: grid  */
    int64_t cells_examined; /* pr_assign: rounded costs the proposal scans
                               examine, from each scan's start column to the
                               column it proposes to (inclusive) or to the
                               row's end; 0 for the other entry points       */
    int64_t barriers;      /* pr_assign: grid (or cluster) barriers the phase
                              loop passed -- one per round of the lowest-index
                              and offset rules, rounds without a proposal
                              included; 0 for the other entry points        */
} pr_stats;

/*
 * Workspace bytes pr_assign needs for an n_rows x n_cols problem
 * (0 if the sizes are invalid).
 */
size_t pr_assign_workspace(int32_t n_rows, int32_t n_cols);

/*
 * pr_assign -- additive approximation of the assignment problem.
 *
 * Defines: Sec. 1 (problem statement; c(M) is the sum of matched costs),
 * Eq. (1) (rounding cbar = eps*floor(c/eps)), Sec. 2.2 (phases: greedy
 * maximal matching on admissible edges, push/evict, dual update; stop when at
 * most eps*|B| vertices of B are free, then match the rest arbitrarily),
 * Sec. 3.3 (unbalanced case |B| <= |A|).  The result's cost is within
 * 3*eps*n_rows of the optimum (Sec. 2.1, Lemma 3.1).
 *
 * The maximal matching of each phase is the deterministic round rule: every
 * still-active free row proposes to its lowest-index admissible column not
 * taken in an earlier round of the phase, each column accepts its
 * lowest-index proposer, rounds repeat until no row proposes.  Completion
 * matches the k-th free row (ascending) with the k-th free column
 * (ascending); duals are left as the main routine ended.
 *
 *   C          n_rows x n_cols costs, dtype dt, leading dimension ldc >= n_cols.
 *              Device memory, or pinned (page-locked) host memory, which the
 *              rounding kernel then reads in place over the host link (the
 *              end-to-end path without a separate copy); other host memory
 *              returns PR_ERR_INVALID before anything is enqueued
 *   eps        0 < eps < 1 with floor(1/eps) <= 32766
 *   n_rows     1 <= n_rows <= n_cols <= 2^24
 *   row_to_col [n_rows] out: column matched to each row (always >= 0)
 *   col_to_row [n_cols] out: row matched to each column, -1 if none
 *   y_row      [n_rows] out: integer duals of the rows (>= 1), units of eps
 *   y_col      [n_cols] out: integer duals of the columns (<= 0), units of eps
 *   cost       [1] out: FP64 sum_i C[i, row_to_col[i]] in input units
 *   stats      host, may be NULL; non-NULL makes the call synchronous
 *   ws, ws_bytes  device workspace, >= pr_assign_workspace(n_rows, n_cols)
 */
pr_status pr_assign(const void *C, pr_dtype dt, int64_t ldc, int32_t n_rows, int32_t n_cols,
                    double eps, int32_t *row_to_col, int32_t *col_to_row, int32_t *y_row,
                    int32_t *y_col, double *cost, pr_stats *stats, void *ws, size_t ws_bytes,
                    void *stream);

/*
 * pr_assign_rule -- pr_assign with a choice of the maximal matching of step
 * (I).  Sec. 2.2 accepts any maximal matching of the admissible graph on the
 * free vertices (the greedy of Lemma 3.4, or Israeli-Itai's randomized one
 * for the parallel bound); every bound of Sec. 2.1 and 3 holds for each.
 *   PR_RULE_LOWEST  pr_assign's rule: every free row proposes to its
 *                   lowest-index admissible column not taken in an earlier
 *                   round of the phase, each column takes its lowest proposer.
 *   PR_RULE_OFFSET  the same rounds, but in phase p (counted from 1) row b
 *                   scans cyclically from column splitmix64(p << 32 | b) mod
 *                   n_cols (SplitMix64's output function, Steele, Lea and
 *                   Flood 2014) and stops after one full turn.  Spreading the
 *                   first proposals over the columns cuts the rounds of a
 *                   phase where most edges are admissible (large eps).
 *   PR_RULE_ISRAELI_ITAI  Israeli and Itai's randomized maximal matching
 *                   (IPL 1986), named by Sec. 3.2 for the O(log n) rounds of
 *                   a phase: per round every live free row and every column
 *                   not yet in M' points to a random admissible neighbour,
 *                   every vertex pointed at keeps one random pointer, every
 *                   vertex picks one of its (at most two) kept edges, and
 *                   edges picked at both ends join M'.  Each random choice
 *                   is the least key (draw >> 24) << 24 | index over the
 *                   candidates, a draw being three SplitMix64 rounds over
 *                   (step, phase, round), the vertex (b, or 2^24 + a for a
 *                   column) and the candidate: deterministic, so the result
 *                   is reproducible.  Every round scans each live row whole.
 *                   Runs on the whole grid (never the cluster form); more
 *                   than 4096 rounds in one phase return
 *                   PR_ERR_NO_CONVERGENCE.
 *   PR_RULE_SEQUENTIAL  the sequential greedy of Sec. 3.2 (the free rows in
 *                   index order, each taking its first admissible column
 *                   not yet in M'), computed without rounds: every free row
 *                   scans on its own, a column goes to the lowest row that
 *                   reaches it in the phase, and a row that loses a column
 *                   to a lower one scans on after it.  The result does not
 *                   depend on the order the scans run in; one grid barrier
 *                   per phase.  stats->rounds counts one round per phase.
 *                   The phase's keys are kept in shared memory, so n_cols
 *                   is at most 196,608 with byte storage (floor(1/eps) <=
 *                   252) and 98,304 otherwise (PR_ERR_INVALID beyond).
 * Other arguments, outputs and errors as pr_assign; cells_examined counts
 * the columns each scan passes.
 */
typedef enum {
    PR_RULE_LOWEST = 0,
    PR_RULE_OFFSET = 1,
    PR_RULE_ISRAELI_ITAI = 2,
    PR_RULE_SEQUENTIAL = 3
} pr_rule;
pr_status pr_assign_rule(pr_rule rule, const void *C, pr_dtype dt, int64_t ldc, int32_t n_rows,
                         int32_t n_cols, double eps, int32_t *row_to_col, int32_t *col_to_row,
                         int32_t *y_row, int32_t *y_col, double *cost, pr_stats *stats, void *ws,
                         size_t ws_bytes, void *stream);

/*
 * pr_assign_staged -- pr_assign for a cost matrix in host memory: the
 * rounding of Eq. 1 overlaps the host-to-device copy.  The rows of C_host go
 * to C_dev in chunks of about 32 MB on a copy stream the library owns (one
 * per device, made on first use), and each chunk is rounded on `stream` as
 * soon as it has arrived, while the next one is being copied; the phase loop
 * then runs as in pr_assign.  The results equal pr_assign(C_dev, ...) bit for
 * bit.
 *
 *   C_host  n_rows x n_cols costs in [0,1] (FP32/FP64), row pitch ldc, host
 *           memory; page-locked (pinned) memory lets the copies run
 *           asynchronously, pageable memory works but each copy then waits
 *           for the host
 *   C_dev   device buffer of the same layout (n_rows rows of pitch ldc), owned
 *           by the caller; it holds the copied costs afterwards (the cost of
 *           the matching is read from it)
 *   other arguments as pr_assign
 * The copy stream first waits for the work already enqueued on `stream`.
 * Enqueueing is serialised across host threads by a library mutex.  Errors
 * as pr_assign; PR_ERR_INVALID also when C_host is not host memory or C_dev
 * not device memory.
 */
pr_status pr_assign_staged(const void *C_host, void *C_dev, pr_dtype dt, int64_t ldc, int32_t n_rows,
                           int32_t n_cols, double eps, int32_t *row_to_col, int32_t *col_to_row,
                           int32_t *y_row, int32_t *y_col, double *cost, pr_stats *stats, void *ws,
                           size_t ws_bytes, void *stream);

/*
 * pr_assign_within -- a matching whose cost is within delta * n_rows of the
 * optimum, for costs in [0, 1].  The main routine of Sec. 2.2 with
 * parameter eps returns a matching within 3 * eps * n_rows of the optimum
 * (Sec. 2.1, Lemma 3.1); the paper's introduction (Sec. 1) gets the
 * eps * n guarantee by running it with eps / 3.  This call does that: it is
 * pr_assign with eps = delta / 3 (one IEEE FP64 division), and the duals it
 * returns are in units of that eps.
 *   delta  0 < delta < 3, with floor(3 / delta) <= 32766
 * Other arguments, outputs and errors as pr_assign.
 */
pr_status pr_assign_within(const void *C, pr_dtype dt, int64_t ldc, int32_t n_rows, int32_t n_cols,
                           double delta, int32_t *row_to_col, int32_t *col_to_row, int32_t *y_row,
                           int32_t *y_col, double *cost, pr_stats *stats, void *ws, size_t ws_bytes,
                           void *stream);

/*
 * pr_dual_bound -- the a-posteriori certificate of a pr_assign solve
 * (Lemma 3.1).  The duals it returns satisfy Eq. (2), y(a) + y(b) <= cbar +
 * eps on every edge; summed over any matching that covers the rows (column
 * duals are <= 0) this gives
 *     L = eps * (sum y_row + sum y_col - n_rows) <= OPT(cbar) <= OPT(c),
 * a lower bound on the optimal cost that needs no optimal solver, so that
 * cost - L bounds the solve's additive error from above.
 *   y_row [n_rows], y_col [n_cols]  the solve's integer duals (units of eps)
 *   eps        the solve's eps
 *   cost       [1] the solve's cost, or NULL
 *   out        [2] out: out[0] = L, out[1] = cost - L (a NaN when cost is NULL)
 * The sums are exact 64-bit integer sums; L is one FP64 product, the gap one
 * FP64 difference.  All pointers are device pointers.  Asynchronous.
 */
pr_status pr_dual_bound(const int32_t *y_row, const int32_t *y_col, int32_t n_rows, int32_t n_cols,
                        double eps, const double *cost, double *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched form: many independent square problems in one persistent launch.  */
/* ------------------------------------------------------------------------ */

/* Launch shape of the batched solver (0 = default). */
typedef struct {
    int32_t threads;     /* threads per solver CTA: 128, 256, 512 or 1024 (0 = 256) */
    int32_t ctas_per_sm; /* resident solver CTAs per SM, 0 = as many as fit        */
} pr_batched_tune;

typedef enum { PR_SQEUCLIDEAN = 0, PR_EUCLIDEAN = 1 } pr_metric;

/*
 * Workspace bytes of pr_assign_batched / pr_assign_batched_points for
 * n_problems problems of sizes n_host[0..n_problems) (host array); 0 if a
 * size is outside 1..5000.
 */
size_t pr_assign_batched_workspace(int32_t n_problems, const int32_t *n_host);

/*
 * pr_assign_batched -- pr_assign's method (Sec. 2.2, Eq. 1, completion of
 * Sec. 2.1) applied to n_problems independent square problems in one
 * persistent launch: one CTA per problem at a time, problems taken largest
 * first, all per-problem state in shared memory.  Each problem's result is
 * bit-identical to pr_assign on that problem alone.
 *
 *   C          packed costs in [0,1]: problem i is n_i x n_i row-major at
 *              element offset sum_{j<i} n_j^2 (rows = the proposing side B)
 *   n_host     host array of the n_i, 1 <= n_i <= 5000
 *   row_to_col, col_to_row, y_row, y_col
 *              packed per problem at offset v_i = sum_{j<i} n_j; indices are
 *              local to the problem (0..n_i-1), duals in units of eps
 *   costs      [n_problems] FP64 matching costs in input units
 *   phases     [n_problems] phases each problem ran
 *   tune       host, may be NULL (defaults)
 *   stats      host, may be NULL; totals over all problems; non-NULL syncs
 * The problem table is copied from host memory with cudaMemcpyAsync, which
 * waits for work queued earlier on `stream`.
 */
pr_status pr_assign_batched(const void *C, pr_dtype dt, int32_t n_problems, const int32_t *n_host,
                            double eps, int32_t *row_to_col, int32_t *col_to_row, int32_t *y_row,
                            int32_t *y_col, double *costs, int64_t *phases,
                            const pr_batched_tune *tune, pr_stats *stats, void *ws,
                            size_t ws_bytes, void *stream);

/*
 * pr_assign_batched_points -- as pr_assign_batched, with the costs of each
 * problem formed from point sets (Sec. 1 and Sec. 5: cost = distance between
 * a point of A and a point of B, scaled so the largest cost is 1).  For
 * problem i, XA and XB hold rows v_i .. v_i + n_i - 1 of (sum n) x dim FP32
 * arrays; XB are the rows (B), XA the columns (A).  d = sum_k (xb_k - xa_k)^2
 * in FP32, one IEEE operation at a time in ascending k (PR_EUCLIDEAN: its
 * IEEE square root); the rounded costs use c = RN32(d / max d).  costs[i] is
 * the matched distance sum in input units, evaluated in FP64.
 */
pr_status pr_assign_batched_points(const float *XA, const float *XB, int32_t dim, pr_metric metric,
                                   int32_t n_problems, const int32_t *n_host, double eps,
                                   int32_t *row_to_col, int32_t *col_to_row, int32_t *y_row,
                                   int32_t *y_col, double *costs, int64_t *phases,
                                   const pr_batched_tune *tune, pr_stats *stats, void *ws,
                                   size_t ws_bytes, void *stream);

/*
 * pr_assign_points -- pr_assign with the costs formed from two point sets on
 * the device instead of read from a stored matrix (Sec. 1: c(a,b) is the
 * distance of a and b; Sec. 5 draws points in the unit square).  XB holds
 * the n_rows row points (the proposing side B) and XA the n_cols column
 * points (A), dim FP32 coordinates each, row-major.  d = sum_k (xb_k -
 * xa_k)^2 in FP32, one IEEE operation at a time in ascending k (PR_EUCLIDEAN:
 * its IEEE square root); the rounded costs of Eq. (1) use c = RN32(d / max d)
 * so that the largest cost is 1.  No n_rows x n_cols input exists: the
 * rounded matrix is written straight into the workspace.
 *   cost       [1] out: the FP64 sum over the rows of the matched d,
 *              re-evaluated in FP64 (input units)
 *   ws, ws_bytes  >= pr_assign_workspace(n_rows, n_cols)
 * Other arguments, outputs and errors as pr_assign.  Coordinates that make
 * a distance non-finite give PR_ERR_INVALID (reported when the call
 * synchronises).
 */
pr_status pr_assign_points(const float *XA, const float *XB, int32_t dim, pr_metric metric, int32_t n_rows,
                           int32_t n_cols, double eps, int32_t *row_to_col, int32_t *col_to_row,
                           int32_t *y_row, int32_t *y_col, double *cost, pr_stats *stats, void *ws,
                           size_t ws_bytes, void *stream);

/*
 * pr_assign_batched_autotune -- picks the batched solver's launch shape for a
 * given batch: runs the solve once per candidate (threads per CTA in {128,
 * 256, 512, 1024} x resident CTAs per SM in {1, 2, 3, 4}; shapes that do not
 * fit are skipped), times each with CUDA events on `stream`, writes the
 * fastest to *best (host) and its time in ms to *best_ms (host), and leaves
 * that shape's results in the outputs.  Points source when XA and XB are both
 * non-NULL (then C and dt are ignored), otherwise the packed matrices C.  Other
 * arguments as pr_assign_batched_points / pr_assign_batched.  Synchronous.
 */
pr_status pr_assign_batched_autotune(const float *XA, const float *XB, int32_t dim, pr_metric metric,
                                     const void *C, pr_dtype dt, int32_t n_problems,
                                     const int32_t *n_host, double eps, int32_t *row_to_col,
                                     int32_t *col_to_row, int32_t *y_row, int32_t *y_col,
                                     double *costs, int64_t *phases, pr_batched_tune *best,
                                     float *best_ms, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Optimal transport (Sec. 4).                                               */
/* ------------------------------------------------------------------------ */

/* Workspace bytes of pr_ot (0 if the sizes are invalid): the rounded costs
 * (n_sup x n_dem, one or two bytes each) and O(n_sup + n_dem) more.  The
 * matched copy counts are kept in one list per demand (32 entries each,
 * plus an arena of 8 (n_sup + n_dem) + 4096 entries for longer lists); a
 * solve whose lists need more arena reports PR_ERR_CAPACITY. */
size_t pr_ot_workspace(int32_t n_sup, int32_t n_dem);

/*
 * pr_ot -- additive approximation of optimal transport (Sec. 4): masses are
 * scaled by theta = 4 max(n_sup, n_dem) / eps, supplies rounded down and
 * demands rounded up to integer copy counts, and the matching algorithm of
 * Sec. 2.2 (unbalanced, Sec. 3.3) runs on the copies with every free supply
 * copy's dual raised to the largest among its siblings.  Copies are handled
 * as clusters (Lemma 4.1: a vertex's copies take at most two dual values).
 * The matched copies give mass(b,a) = copies / theta; a demand that received
 * more than its mass gives the excess back from its highest-index supplier,
 * and every supply's remainder is routed north-west-corner style (supplies
 * ascending, demands ascending) into the remaining demand capacity.  The
 * paper leaves this fix-up to another paper; here the remainders are first
 * rounded down to whole units of 2^-62 and the rule runs on exact integers
 * (each supply loses less than 2^-62 of its mass).
 *
 *   C           n_sup x n_dem costs in [0,1] (rows = supplies B), ldc >= n_dem
 *   supply      [n_sup] FP64 masses nu >= 0 summing to 1 (device)
 *   demand      [n_dem] FP64 masses mu >= 0 summing to 1 (device); the
 *               demand must cover the supply (else PR_ERR_NO_CONVERGENCE).
 *               PR_ERR_INVALID for a negative or NaN mass, a mass >= 2, or
 *               a side whose floor(m 2^32) sum to 1.5 * 2^32 or more
 *   plan_row, plan_col, plan_mass  [plan_cap] out: the plan as (supply,
 *               demand, mass) triples, each pair at most once
 *   plan_nnz    [1] out: number of triples (also written when > plan_cap,
 *               which is PR_ERR_CAPACITY)
 *   y_sup       [n_sup] out: dual of the free copies of each supply (its
 *               largest copy dual), units of eps
 *   dem_kmin, dem_lo, dem_hi  [n_dem] out: each demand's copies have duals
 *               -dem_kmin (dem_lo copies) and -dem_kmin - 1 (dem_hi copies)
 *   cost        [1] out: sum of mass * C over the plan (FP64)
 *   stats       host, may be NULL
 * Like pr_assign, pr_ot only enqueues work on `stream` and synchronises it
 * iff `stats` is non-NULL; the plan size and every device-side error
 * (invalid masses or costs, the loop's time-out or phase cap, the plan
 * exceeding plan_cap, the list arena running out) are found on the device.
 * With stats == NULL, pr_ws_status(ws, stream) reports them later.
 */
pr_status pr_ot(const void *C, pr_dtype dt, int64_t ldc, int32_t n_sup, int32_t n_dem,
                const double *supply, const double *demand, double eps, int64_t plan_cap,
                int32_t *plan_row, int32_t *plan_col, double *plan_mass, int64_t *plan_nnz,
                int32_t *y_sup, int32_t *dem_kmin, int32_t *dem_lo, int32_t *dem_hi, double *cost,
                pr_stats *stats, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Differentiation of the assignment loss.                                   */
/* ------------------------------------------------------------------------ */

/*
 * pr_assign_backward -- gradient of the squared-Euclidean assignment loss
 *   L_p = (1/n) sum_i |x_i - y_sigma(i)|^2
 * for `batch` pairs of point clouds with the plans sigma_p held fixed (the
 * plan of Sec. 2.2 is piecewise constant in the coordinates, so this is the
 * gradient wherever the plan is locally unique; the paper has no backward
 * pass, this is the envelope rule applied to its output).
 *
 *   row_to_col [batch][n] completed plans (permutations), e.g. the packed
 *              output of pr_assign_batched_points on the pairs
 *   X, Y       [batch][n][dim] FP32 rows (B) and columns (A) of each pair
 *   grad_cost  [batch] incoming gradient of each L_p
 *   grad_X     [batch][n][dim] out: g * 2 (x_i - y_sigma(i)) / n
 *   grad_Y     [batch][n][dim] out: minus that, at row sigma(i)
 *   grad_C     [batch][n][n] out or NULL: g / n on matched entries, else 0
 * Each value is formed in FP64 as ((x - y) * 2) / n * g and rounded once.
 * Asynchronous; the plans must be permutations (not checked on the device).
 */
pr_status pr_assign_backward(const int32_t *row_to_col, const float *X, const float *Y,
                             int32_t batch, int32_t n, int32_t dim, const float *grad_cost,
                             float *grad_X, float *grad_Y, float *grad_C, void *stream);

/*
 * pr_assign_noalloc -- pr_assign for callers that cannot allocate device
 * memory: code running where cudaMalloc is not allowed or not wanted (while
 * a stream is being captured into a CUDA graph, inside a host application
 * that forbids device allocations after start-up, or in a latency-critical
 * loop that must not enter the allocator), and callers with no way to keep
 * a workspace between calls.  It computes exactly what pr_assign computes.
 * The paper has no counterpart: this is a packaging of the same solve.
 *
 * Instead of a caller workspace it uses one device array of 2.25 MiB built
 * into the library; every GPU that loads the library holds that array until
 * the process exits.  Limits: n_rows <= n_cols <= 1024 (larger sizes return
 * PR_ERR_INVALID with a message).  Every call looks up the array's device
 * address (cudaGetSymbolAddress, with the call's device current), and the
 * first call on a device is also where the runtime loads the library's
 * kernels on it: make that first call before any stream capture.  All calls
 * on a device share the array and each call reinitialises what it uses, so
 * calls that overlap on the GPU (other streams, other host threads) race:
 * serialise them.  No memory is allocated or freed by this call.  C is
 * checked as in pr_assign (device, managed or pinned host memory; other host
 * memory is refused with PR_ERR_INVALID before anything is enqueued).  Other
 * arguments and errors as pr_assign, with one difference: a device-side
 * error (a spin-limit time-out, an internal check) is returned only when
 * stats != NULL, which makes the call synchronous; with stats == NULL such
 * an error goes unreported, since the array's status word has no query.
 */
pr_status pr_assign_noalloc(const void *C, pr_dtype dt, int64_t ldc, int32_t n_rows, int32_t n_cols,
                            double eps, int32_t *row_to_col, int32_t *col_to_row, int32_t *y_row,
                            int32_t *y_col, double *cost, pr_stats *stats, void *stream);

/*
 * Synchronise `stream` and return the device-side status recorded in a
 * workspace by the last call that used it (PR_OK if none).  For callers that
 * pass stats == NULL.  `ws` must be a workspace of that call.
 */
pr_status pr_ws_status(const void *ws, void *stream);

/*
 * Profiling hook (thread-local).  When `start` and `stop` are cudaEvent_t
 * handles, each later solver call made by this thread records `start` right
 * before and `stop` right after its dominant kernel (the persistent phase
 * kernel) on the call's stream, so a caller can time that kernel alone with
 * CUDA events.  Pass NULL, NULL to stop.  The events are borrowed, not owned.
 */
void pr_set_kernel_events(void *start, void *stop);

/*
 * pr_probe_latency -- the measured floors under one round of the phase loop
 * on the current device: *barrier_ns, the mean time of one grid barrier of
 * the kind the phase kernel uses (one CTA of 512 threads per SM, a release
 * reduction and acquire polls, 2000 in a row), and *l2_ns, the mean time of
 * one dependent load that hits L2 (a chain of 4096 loads through a 4 MB
 * permutation).  Diagnostics for a latency roofline; the paper has no
 * counterpart.  `ws` is device memory of at least pr_probe_workspace()
 * bytes, 256-byte aligned, owned by the caller.  Synchronises `stream`.
 * Errors: PR_ERR_WORKSPACE, PR_ERR_CUDA, PR_ERR_TIMEOUT (a barrier wait ran
 * out).
 */
size_t pr_probe_workspace(void);
pr_status pr_probe_latency(void *ws, size_t ws_bytes, double *barrier_ns, double *l2_ns, void *stream);

/* Thread-local text of the last error (never NULL). */
const char *pr_last_error(void);

/* Name of a status code. */
const char *pr_status_string(pr_status s);

#ifdef __cplusplus
}
#endif
#endif /* PROT_H */
