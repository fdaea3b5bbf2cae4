// points.cuh -- costs from point sets, shared by the single-problem and the
// batched solvers.  d(b,a) = sum_k (xb_k - xa_k)^2 in FP32, one IEEE
// operation at a time in ascending k (no contraction); Euclidean takes the
// IEEE square root.  The rounded costs use c = RN32(d / max d), so the largest
// cost is 1 (Sec. 1); reported costs re-evaluate the matched d in FP64.
#pragma once

namespace prot {
namespace {

__device__ __forceinline__ float dist_f32(const float *xb, const float *xa, int dim, int squared) {
    float acc = 0.0f;
    for (int k = 0; k < dim; ++k) {
        const float t = __fsub_rn(xb[k], xa[k]);
        const float sq = __fmul_rn(t, t);
        acc = k == 0 ? sq : __fadd_rn(acc, sq);
    }
    return squared ? acc : __fsqrt_rn(acc);
}

__device__ __forceinline__ double dist_f64(const float *xb, const float *xa, int dim, int squared) {
    double acc = 0.0;
    for (int k = 0; k < dim; ++k) {
        const double t = __dsub_rn((double)xb[k], (double)xa[k]);
        const double sq = __dmul_rn(t, t);
        acc = k == 0 ? sq : __dadd_rn(acc, sq);
    }
    return squared ? acc : __dsqrt_rn(acc);
}

}  // namespace
}  // namespace prot
