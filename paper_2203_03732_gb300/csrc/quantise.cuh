// quantise.cuh -- the rounding kernel of Eq. (1), shared by the single-
// problem and the optimal-transport paths.
#pragma once

#include "prot_internal.cuh"
#include "scan_common.cuh"

namespace prot {
namespace {

// ---------------------------------------------------------------------------
// k_quantise: Eq. (1) exactly (quantise_one), 8 columns per thread.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_quantise(const T *__restrict__ C, long long ldc, int nB, int nA, int ldq,
                           double eps, float inv_eps, uint16_t *__restrict__ cb, WsHead *head) {
    const int groups = ldq >> 3;
    const long long total = (long long)nB * groups;
    bool bad = false;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(g / groups);
        const int a0 = (int)(g - (long long)b * groups) << 3;
        const T *row = C + (long long)b * ldc;
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t h[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int a = a0 + 2 * j + k;
                if (a < nA) {
                    const double c = (double)row[a];
                    if (!(c >= 0.0 && c <= 1.0)) {
                        bad = true;
                        h[k] = 0;
                    } else {
                        h[k] = quantise_one(c, eps, inv_eps);
                    }
                } else {
                    h[k] = kPadCost;
                }
            }
            w[j] = h[0] | (h[1] << 16);
        }
        *reinterpret_cast<uint4 *>(cb + (long long)b * ldq + a0) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (bad) record_error(head, PR_ERR_INVALID);
}

}  // namespace
}  // namespace prot
