// certificate.cu -- pr_dual_bound: the a-posteriori certificate of a solve.
//
// Lemma 3.1: when the main routine stops, every edge satisfies Eq. (2),
// y(a) + y(b) <= cbar(a,b) + eps.  Sum it over the edges of any matching M*
// that covers the rows: sum_{M*} cbar >= sum_b y(b) + sum_{a in M*} y(a) -
// eps n_B, and every column dual is <= 0, so adding the columns M* leaves out
// only lowers the right side.  Hence
//     L = eps * (sum_b y_b + sum_a y_a - n_B) <= OPT(cbar) <= OPT(c)
// (cbar <= c by Eq. 1), with the duals as the integers the solver keeps (units
// of eps).  L needs no optimal solver, and c(M) - L bounds the additive error
// of the returned matching from above.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "prot_internal.cuh"

namespace prot {
namespace {

constexpr int kThreads = 1024;

// One CTA: the exact 64-bit integer sum of both dual vectors (integers, so
// the order of the additions does not matter), then L and the gap.
__global__ void __launch_bounds__(kThreads)
k_dual_bound(const int32_t *__restrict__ y_row, const int32_t *__restrict__ y_col, int n_rows,
             int n_cols, double eps, const double *__restrict__ cost, double *__restrict__ out) {
    __shared__ long long part[kThreads / 32];
    long long s = 0;
    for (int i = threadIdx.x; i < n_rows; i += kThreads) s += y_row[i];
    for (int i = threadIdx.x; i < n_cols; i += kThreads) s += y_col[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += part[w];
        const double L = __dmul_rn(eps, (double)(t - (long long)n_rows));  // |t| < 2^53: exact
        out[0] = L;
        out[1] = cost ? __dsub_rn(*cost, L) : __longlong_as_double(0x7FF8000000000000ll);
    }
}

}  // namespace
}  // namespace prot

using namespace prot;

extern "C" pr_status pr_dual_bound(const int32_t *y_row, const int32_t *y_col, int32_t n_rows,
                                   int32_t n_cols, double eps, const double *cost, double *out,
                                   void *stream) {
    if (!y_row || !y_col || !out) return fail(PR_ERR_INVALID, "pr_dual_bound: NULL pointer argument");
    if (n_rows < 1 || n_cols < n_rows) return fail(PR_ERR_INVALID, "pr_dual_bound: need 1 <= n_rows <= n_cols");
    if (!(eps > 0.0 && eps < 1.0)) return fail(PR_ERR_INVALID, "pr_dual_bound: need 0 < eps < 1");
    k_dual_bound<<<1, kThreads, 0, (cudaStream_t)stream>>>(y_row, y_col, n_rows, n_cols, eps, cost, out);
    PR_CUDA(cudaGetLastError());
    return PR_OK;
}
