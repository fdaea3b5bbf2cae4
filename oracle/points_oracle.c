/*
 * points_oracle.c -- oracle for the point-cloud forms (batched solver and the
 * differentiable assignment loss).  TEST INFRASTRUCTURE ONLY; shares nothing
 * with the CUDA library.
 *
 * Costs from points (the cost c(a,b) of Sec. 1, for point sets A and B):
 *   d(b,a) = sum_k (xb_k - xa_k)^2 in FP32, one IEEE operation at a time in
 *            ascending k (no fused multiply-add); plain Euclidean takes the
 *            IEEE square root of that sum.
 *   M      = max over all pairs of d;  c = RN32(d / M)  (0 when M == 0), so the
 *            largest cost is 1 as Sec. 1 assumes.
 * The reported matching cost is in input units: sum over matched pairs of d
 * evaluated in FP64 (coordinates widened exactly, same order), summed with
 * Neumaier compensation in ascending row order.
 *
 * Gradient of the loss L = (g/n) sum_i d(x_i, y_sigma(i)) for squared
 * Euclidean d, holding the plan sigma fixed (the plan is piecewise constant in
 * the coordinates, so this is the gradient wherever the plan is locally
 * unique): dL/dx_i = g * 2 (x_i - y_sigma(i)) / n, dL/dy_j = -g * 2 (x_i -
 * y_j) / n for sigma(i) = j, each evaluated in FP64 as ((x - y) * 2) / n * g
 * and rounded once to FP32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "prot_oracle.h"

static float dist_f32(const float *xb, const float *xa, int32_t dim, int squared)
{
    float acc = 0.0f;
    for (int32_t k = 0; k < dim; ++k) {
        float t = xb[k] - xa[k];
        float sq = t * t;
        acc = (k == 0) ? sq : acc + sq;
    }
    return squared ? acc : sqrtf(acc);
}

static double dist_f64(const float *xb, const float *xa, int32_t dim, int squared)
{
    double acc = 0.0;
    for (int32_t k = 0; k < dim; ++k) {
        double t = (double)xb[k] - (double)xa[k];
        double sq = t * t;
        acc = (k == 0) ? sq : acc + sq;
    }
    return squared ? acc : sqrt(acc);
}

/* Normalised FP32 costs C[b][a] (row-major nB x nA) from points. */
void or_points_cost(const float *XA, const float *XB, int32_t nA, int32_t nB, int32_t dim,
                    int32_t squared, float *C)
{
    float M = 0.0f;
    for (int32_t b = 0; b < nB; ++b)
        for (int32_t a = 0; a < nA; ++a) {
            float d = dist_f32(XB + (int64_t)b * dim, XA + (int64_t)a * dim, dim, squared);
            C[(int64_t)b * nA + a] = d;
            if (d > M) M = d;
        }
    for (int64_t i = 0; i < (int64_t)nB * nA; ++i)
        C[i] = (M > 0.0f) ? C[i] / M : 0.0f;
}

/* FP64 matching cost in input units. */
double or_points_match_cost(const float *XA, const float *XB, int32_t nB, int32_t dim,
                            int32_t squared, const int32_t *row_to_col)
{
    double s = 0.0, comp = 0.0;
    for (int32_t b = 0; b < nB; ++b) {
        double x = dist_f64(XB + (int64_t)b * dim, XA + (int64_t)row_to_col[b] * dim, dim, squared);
        double t = s + x;
        if (fabs(s) >= fabs(x)) comp += (s - t) + x;
        else comp += (x - t) + s;
        s = t;
    }
    return s + comp;
}

/* One point-cloud problem: costs from points, Eq. (1), the Sec. 2.2 main
 * routine, completion, cost in input units. */
int or_assign_points(const float *XA, const float *XB, int32_t nA, int32_t nB, int32_t dim,
                     int32_t squared, double eps, int32_t *match_b, int32_t *match_a,
                     int32_t *y_b, int32_t *y_a, double *cost, or_stats *st)
{
    if (nB < 1 || nA < nB || dim < 1) return OR_ERR_INVALID;
    float *C = (float *)malloc(sizeof(float) * (size_t)nB * (size_t)nA);
    int32_t *cb = (int32_t *)malloc(sizeof(int32_t) * (size_t)nB * (size_t)nA);
    if (!C || !cb) { free(C); free(cb); return OR_ERR_NOMEM; }
    or_points_cost(XA, XB, nA, nB, dim, squared, C);
    int rc = or_quantise_f32(C, nA, nB, nA, eps, cb);
    if (rc == 0) {
        int32_t T = or_threshold(eps, nB);
        rc = or_assign_int(cb, nB, nA, T, 0, or_phase_cap(eps, nB), match_b, match_a, y_b, y_a,
                           st, NULL, 0);
    } else {
        rc = OR_ERR_INVALID;
    }
    free(C);
    free(cb);
    if (rc != OR_OK) return rc;
    or_complete(nB, nA, match_b, match_a);
    *cost = or_points_match_cost(XA, XB, nB, dim, squared, match_b);
    return OR_OK;
}

/* Gradient of (g/n) * sum_i |x_i - y_sigma(i)|^2 w.r.t. X (rows) and Y (cols). */
void or_sqeuclid_backward(const float *X, const float *Y, int32_t n, int32_t dim,
                          const int32_t *row_to_col, float g, float *gX, float *gY)
{
    memset(gY, 0, sizeof(float) * (size_t)n * dim);
    for (int32_t i = 0; i < n; ++i) {
        int32_t j = row_to_col[i];
        for (int32_t k = 0; k < dim; ++k) {
            double t = (double)X[(int64_t)i * dim + k] - (double)Y[(int64_t)j * dim + k];
            double v = ((t * 2.0) / (double)n) * (double)g;
            gX[(int64_t)i * dim + k] = (float)v;
            gY[(int64_t)j * dim + k] = (float)(-v);
        }
    }
}
