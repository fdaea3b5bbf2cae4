// backward.cu -- pr_assign_backward: gradients of the assignment loss.
//
// For each pair p of point clouds X_p (rows, the proposing side B) and Y_p
// (columns, A) with plan sigma_p (row_to_col), the loss is
//   L_p = (1/n) sum_i |x_i - y_sigma(i)|^2        (squared Euclidean, input units)
// and the plan is held fixed (it is piecewise constant in the coordinates;
// where it is locally unique this is the gradient).  With g_p the incoming
// gradient of L_p:
//   dL/dx_i = g_p * 2 (x_i - y_sigma(i)) / n,   dL/dy_sigma(i) = -dL/dx_i,
//   dL/dC[i, j] = g_p / n if j = sigma(i), else 0   (optional).
// Each component is evaluated in FP64 as ((x - y) * 2) / n * g with IEEE
// operations in that order and rounded once to FP32.  A completed plan is a
// permutation, so every gradient entry has exactly one writer.
#include <cuda_runtime.h>
#include <stdint.h>

#include "prot_internal.cuh"

namespace prot {
namespace {

__global__ void k_backward(const int32_t *__restrict__ r2c, const float *__restrict__ X,
                           const float *__restrict__ Y, int batch, int n, int dim,
                           const float *__restrict__ g, float *__restrict__ gX,
                           float *__restrict__ gY) {
    const long long total = (long long)batch * n;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(t / n);
        const int j = r2c[t];
        if (j < 0 || j >= n) continue;  // not a completed plan: entries left unwritten
        const double gp = (double)g[p];
        const float *x = X + t * dim;
        const float *y = Y + ((long long)p * n + j) * dim;
        float *gx = gX + t * dim;
        float *gy = gY + ((long long)p * n + j) * dim;
        for (int k = 0; k < dim; ++k) {
            const double d = __dsub_rn((double)x[k], (double)y[k]);
            const double v = __dmul_rn(__ddiv_rn(__dmul_rn(d, 2.0), (double)n), gp);
            gx[k] = __double2float_rn(v);
            gy[k] = __double2float_rn(-v);
        }
    }
}

__global__ void k_grad_c(const int32_t *__restrict__ r2c, int batch, int n,
                         const float *__restrict__ g, float *__restrict__ gC) {
    const long long total = (long long)batch * n * n;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long pi = t / n;  // pair * n + row
        const int j = (int)(t - pi * n);
        const int p = (int)(pi / n);
        gC[t] = r2c[pi] == j ? __double2float_rn(__ddiv_rn((double)g[p], (double)n)) : 0.0f;
    }
}

}  // namespace
}  // namespace prot

using namespace prot;

extern "C" pr_status pr_assign_backward(const int32_t *row_to_col, const float *X, const float *Y,
                                        int32_t batch, int32_t n, int32_t dim,
                                        const float *grad_cost, float *grad_X, float *grad_Y,
                                        float *grad_C, void *stream) {
    if (!row_to_col || !X || !Y || !grad_cost || !grad_X || !grad_Y)
        return fail(PR_ERR_INVALID, "pr_assign_backward: NULL pointer argument");
    if (batch < 1 || n < 1 || dim < 1 || dim > 4096)
        return fail(PR_ERR_INVALID, "pr_assign_backward: need batch, n >= 1 and 1 <= dim <= 4096");
    cudaStream_t st = (cudaStream_t)stream;
    const DeviceInfo &di = device_info();
    const long long rows = (long long)batch * n;
    const int grid = (int)((rows + 255) / 256 < (long long)di.sms * 8 ? (rows + 255) / 256 : di.sms * 8);
    k_backward<<<grid, 256, 0, st>>>(row_to_col, X, Y, batch, n, dim, grad_cost, grad_X, grad_Y);
    PR_CUDA(cudaGetLastError());
    if (grad_C) {
        const long long cells = rows * n;
        const int g2 = (int)((cells + 255) / 256 < (long long)di.sms * 16 ? (cells + 255) / 256 : di.sms * 16);
        k_grad_c<<<g2, 256, 0, st>>>(row_to_col, batch, n, grad_cost, grad_C);
        PR_CUDA(cudaGetLastError());
    }
    return PR_OK;
}
