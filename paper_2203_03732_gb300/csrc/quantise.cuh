// quantise.cuh -- the rounding kernel of Eq. (1), shared by the single-
// problem and the optimal-transport paths.
#pragma once

#include "prot_internal.cuh"
#include "scan_common.cuh"

namespace prot {
namespace {

// ---------------------------------------------------------------------------
// k_quantise: Eq. (1) exactly, 8 columns per thread, one 16-byte store.  With
// VEC the row's 8 costs are read with 16-byte loads (rows 16-byte aligned).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t quantise_elem(const double *row, int a, const EpsSplit &e) {
    const unsigned long long bits = __double_as_longlong(row[a]);
    return quantise_bits((uint32_t)(bits >> 32), (uint32_t)bits, e);
}
__device__ __forceinline__ uint32_t quantise_elem(const float *row, int a, const EpsSplit &e) {
    return quantise_fbits(__float_as_uint(row[a]), e);
}

// CB is the stored type: uint16_t, or uint8_t when every cbar <= 252 (the
// caller checks floor(1/eps) <= 252); padding columns get 0x7FFF / 0xFF.
template <class T, bool VEC, class CB>
__global__ void k_quantise(const T *__restrict__ C, long long ldc, int nB, int nA, int ldq,
                           EpsSplit e, CB *__restrict__ cb, WsHead *head) {
    constexpr uint32_t kPad = sizeof(CB) == 1 ? 0xFFu : (uint32_t)kPadCost;
    // Grid-stride over (row, group of 8 columns); the row and group indices
    // advance by the stride's quotient and remainder (no division per step).
    const int groups = ldq >> 3;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long g0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int step_b = (int)(stride / groups), step_g = (int)(stride % groups);
    int b = (int)(g0 / groups), gi = (int)(g0 % groups);
    bool bad = false;
    for (; b < nB; b += step_b, gi += step_g) {
        if (gi >= groups) {
            gi -= groups;
            ++b;
            if (b >= nB) break;
        }
        const int a0 = gi << 3;
        const T *row = C + (long long)b * ldc;
        uint32_t h[8];
        if (VEC && a0 + 8 <= nA) {
            // 8 consecutive costs: 4 x 16 B (FP64) or 2 x 16 B (FP32)
            if (sizeof(T) == 8) {
                const uint4 *v = reinterpret_cast<const uint4 *>(row + a0);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint4 x = __ldg(v + j);
                    h[2 * j] = quantise_bits(x.y, x.x, e);
                    h[2 * j + 1] = quantise_bits(x.w, x.z, e);
                }
            } else {
                const uint4 *v = reinterpret_cast<const uint4 *>(row + a0);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const uint4 x = __ldg(v + j);
                    h[4 * j] = quantise_fbits(x.x, e);
                    h[4 * j + 1] = quantise_fbits(x.y, e);
                    h[4 * j + 2] = quantise_fbits(x.z, e);
                    h[4 * j + 3] = quantise_fbits(x.w, e);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                h[j] = a0 + j < nA ? quantise_elem(row, a0 + j, e) : kPad;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (h[j] == 0xFFFFFFFFu) {
                bad = true;
                h[j] = 0;
            }
        }
        if (sizeof(CB) == 1) {
            *reinterpret_cast<uint2 *>(cb + (long long)b * ldq + a0) =
                make_uint2(h[0] | (h[1] << 8) | (h[2] << 16) | (h[3] << 24),
                           h[4] | (h[5] << 8) | (h[6] << 16) | (h[7] << 24));
        } else {
            *reinterpret_cast<uint4 *>(cb + (long long)b * ldq + a0) =
                make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
        }
    }
    if (bad) record_error(head, PR_ERR_INVALID);
}

// Launch k_quantise with 16-byte loads when every row starts 16-byte aligned.
template <class T, class CB = uint16_t>
void launch_quantise(const T *C, long long ldc, int nB, int nA, int ldq, double eps, CB *cb,
                     WsHead *head, int grid, cudaStream_t st) {
    const EpsSplit e = make_eps_split(eps);
    const bool vec = ((uintptr_t)C % 16 == 0) && ((ldc * (long long)sizeof(T)) % 16 == 0);
    if (vec) k_quantise<T, true, CB><<<grid, 256, 0, st>>>(C, ldc, nB, nA, ldq, e, cb, head);
    else k_quantise<T, false, CB><<<grid, 256, 0, st>>>(C, ldc, nB, nA, ldq, e, cb, head);
}

}  // namespace
}  // namespace prot
