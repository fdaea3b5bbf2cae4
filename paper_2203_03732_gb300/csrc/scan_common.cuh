// scan_common.cuh -- device primitives shared by the single-problem and the
// batched solvers: exact rounding of Eq. (1), the packed 16-bit admissibility
// test, the per-column proposal word and a few load forms.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace prot {

constexpr uint16_t kPadCost = 0x7FFF;  // cbar of padding columns
constexpr uint16_t kPadKey = 0x8000;   // k of padding columns: pad sum 0xFFFF never matches

// Eq. (1) exactly: the largest k with k * eps <= c, for 0 <= c <= 1.
// An FP32 estimate q of c/eps is within 0.006 of the exact quotient (three
// roundings of relative size 2^-24 on a quotient <= 32767), so floor(q) is
// exact whenever q is at least 1/64 away from an integer.  Otherwise the
// integer is settled with fma(-k, eps, c), whose sign is that of the exact
// c - k*eps.  No FP64 division runs per element.
__device__ __forceinline__ uint32_t quantise_one(double c, double eps, float inv_eps) {
    const float q = __fmul_rn((float)c, inv_eps);
    const float kf = floorf(q);
    const float fr = q - kf;
    int k = (int)kf;
    if (!(fr >= 0.015625f && fr <= 0.984375f)) {
        while (k > 0 && fma(-(double)k, eps, c) < 0.0) --k;
        while (fma(-(double)(k + 1), eps, c) >= 0.0) ++k;
    }
    return (uint32_t)k;
}

// Bit j of the result: 16-bit lane j of the 8-lane vector s equals t (t2 =
// t in both halves).
__device__ __forceinline__ unsigned eq_mask(uint4 s, uint32_t t2) {
    const uint32_t w0 = s.x ^ t2, w1 = s.y ^ t2, w2 = s.z ^ t2, w3 = s.w ^ t2;
    unsigned m = 0;
    m |= (w0 & 0xFFFFu) == 0 ? 1u : 0u;
    m |= (w0 >> 16) == 0 ? 2u : 0u;
    m |= (w1 & 0xFFFFu) == 0 ? 4u : 0u;
    m |= (w1 >> 16) == 0 ? 8u : 0u;
    m |= (w2 & 0xFFFFu) == 0 ? 16u : 0u;
    m |= (w2 >> 16) == 0 ? 32u : 0u;
    m |= (w3 & 0xFFFFu) == 0 ? 64u : 0u;
    m |= (w3 >> 16) == 0 ? 128u : 0u;
    return m;
}

// Read-only 16-byte load that does not allocate in L1 (streamed rows).
__device__ __forceinline__ uint4 ld_nc_na_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Proposal word of a column: (round << 32) | (0xFFFFFFFF - row).  An
// atomicMax keeps the lowest row among same-round proposals and lets a later
// round overwrite an earlier one.  Round 0 with row -1 means "never won".
__device__ __forceinline__ unsigned tag_of(unsigned long long w) { return (unsigned)(w >> 32); }
__device__ __forceinline__ int row_of(unsigned long long w) { return (int)(0xFFFFFFFFu - (unsigned)w); }
__device__ __forceinline__ unsigned long long word_of(unsigned R, int b) {
    return ((unsigned long long)R << 32) | (0xFFFFFFFFu - (unsigned)b);
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace prot
