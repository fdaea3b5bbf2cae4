// scan_common.cuh -- device primitives shared by the single-problem and the
// batched solvers: exact rounding of Eq. (1), the packed 16-bit admissibility
// test, the per-column proposal word and a few load forms.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

namespace prot {

constexpr uint16_t kPadCost = 0x7FFF;  // cbar of padding columns
constexpr uint16_t kPadKey = 0x8000;   // k of padding columns: pad sum 0xFFFF never matches

// eps split exactly as me * 2^ee (me < 2^53, an integer), plus the FP32
// reciprocal used for the estimate and the estimate's margin.  Built on the
// host by make_eps_split.
struct EpsSplit {
    unsigned long long me;
    int ee;
    float inv;
    float win;  // an estimate within win of an integer takes the exact test
};

// The FP32 estimate q of c / eps (c truncated to 24 significant bits:
// relative error < 2^-23; RN32(1/eps) and the rounded product: 2^-24 each)
// is within c / eps * 2^-22 (1 + 2^-24) < (floor(1/eps) + 1) * 2^-22 of the
// exact quotient, as c <= 1.  The margin is twice that, at most 1/64: at
// eps = 0.01 it is 5e-5, so about one cost in 10^4 takes the exact test.
inline EpsSplit make_eps_split(double eps) {  // eps normal, in (0, 1)
    unsigned long long bits;
    memcpy(&bits, &eps, sizeof bits);
    EpsSplit e;
    e.me = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    e.ee = (int)((bits >> 52) & 0x7FF) - 1075;
    e.inv = (float)(1.0 / eps);
    const double w = (floor(1.0 / eps) + 1.0) * ldexp(1.0, -21);
    e.win = (float)(w < 0.015625 ? w : 0.015625);
    return e;
}

// Exact test c >= m * eps for c = mc * 2^ec (mc < 2^53) and 1 <= m < 2^16,
// in 128-bit integer arithmetic: both sides are brought to the smaller
// exponent and compared.  Outside the shifts that fit in 128 bits the
// answer follows from the exponents alone (c is normal, so 2^23 <= mc for
// FP32 and 2^52 <= mc for FP64; 2^52 <= m * me < 2^69).
__device__ __forceinline__ bool ge_multiple(unsigned long long mc, int ec, uint32_t m, const EpsSplit &e) {
    const int d = ec - e.ee;
    if (d > 74) return true;
    if (d < -58) return false;
    unsigned __int128 lhs = mc, rhs = (unsigned __int128)e.me * m;
    if (d >= 0) lhs <<= d;
    else rhs <<= -d;
    return lhs >= rhs;
}

// Eq. (1) exactly: cbar = the largest k with k * eps <= c, for 0 <= c <= 1.
// An FP32 estimate q of c/eps is within (floor(1/eps) + 1) * 2^-22 of the
// exact quotient (see make_eps_split), so floor(q) is exact whenever q is at
// least e.win (twice that bound, at most 1/64) away from an integer.
// Otherwise the exact quotient lies within 1/32 of the integer m nearest q,
// so the floor is m or m - 1, settled by the exact integer test c >= m * eps.
// No floating-point division and no FP64 instruction runs (GB300 runs FP64
// at a small fraction of its FP32 rate).
//
// For an FP64 cost given by its bit pattern.  Range test on the bits:
// 0 <= c <= 1 (or -0.0), which also rejects NaN and infinities.  The FP32
// estimate truncates the mantissa (relative error < 2^-23) before the two
// roundings of the product.
// Returns 0xFFFFFFFF for a cost outside [0, 1].
__device__ __forceinline__ uint32_t quantise_bits(uint32_t hi, uint32_t lo, const EpsSplit &e) {
    if (hi >= 0x80000000u) {  // sign bit: only -0.0 is valid
        return (hi == 0x80000000u && lo == 0u) ? 0u : 0xFFFFFFFFu;
    }
    if (hi > 0x3FF00000u || (hi == 0x3FF00000u && lo != 0u)) return 0xFFFFFFFFu;  // > 1, NaN, inf
    const uint32_t ex = hi >> 20;
    if (ex <= 896u) {
        // c < 2^-126 (zero or tiny): floor(c / eps) is 0 unless eps is tinier,
        // which eps >= 1/32767 rules out
        return 0u;
    }
    const uint32_t fbits = ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const float q = __fmul_rn(__uint_as_float(fbits), e.inv);
    const float kf = floorf(q);
    const float fr = q - kf;
    uint32_t k = (uint32_t)kf;
    if (!(fr >= e.win && fr <= 1.0f - e.win)) {
        const uint32_t m = k + (fr > 0.5f ? 1u : 0u);
        if (m == 0u) return 0u;
        const unsigned long long mc = (((unsigned long long)(hi & 0xFFFFFu) << 32) | lo) | (1ull << 52);
        k = ge_multiple(mc, (int)ex - 1075, m, e) ? m : m - 1u;
    }
    return k;
}

// The same for an FP32 cost: range test on the bits, exact FP32 estimate,
// the same integer test near a multiple of eps.
__device__ __forceinline__ uint32_t quantise_fbits(uint32_t fb, const EpsSplit &e) {
    if (fb >= 0x80000000u) return fb == 0x80000000u ? 0u : 0xFFFFFFFFu;
    if (fb > 0x3F800000u) return 0xFFFFFFFFu;
    const uint32_t ex = fb >> 23;
    if (ex == 0u) return 0u;  // zero or subnormal: below eps >= 1/32767
    const float q = __fmul_rn(__uint_as_float(fb), e.inv);
    const float kf = floorf(q);
    const float fr = q - kf;
    uint32_t k = (uint32_t)kf;
    if (!(fr >= e.win && fr <= 1.0f - e.win)) {
        const uint32_t m = k + (fr > 0.5f ? 1u : 0u);
        if (m == 0u) return 0u;
        const unsigned long long mc = (unsigned long long)((fb & 0x7FFFFFu) | 0x800000u);
        k = ge_multiple(mc, (int)ex - 150, m, e) ? m : m - 1u;
    }
    return k;
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

// Byte form of the test on four packed bytes: 0x80 in each byte i with
// c_i + k_i == t (t4 = t in all four bytes), else 0.  The low seven bits of
// each byte are added with no carry into the next byte and bit 7 by
// exclusive or, which gives every byte's sum mod 256; a byte whose true sum
// reaches 256 (carry out of its bit 7) is masked out, since such a sum never
// equals a target <= 253.  The zero test of z = sum ^ t4 is exact per byte:
// (z & 0x7F) + 0x7F sets bit 7 iff the low seven bits are not all zero.
__device__ __forceinline__ uint32_t byte_marks(uint32_t c, uint32_t k, uint32_t t4) {
    const uint32_t s7 = (c & 0x7F7F7F7Fu) + (k & 0x7F7F7F7Fu);  // bit 7: carry out of bits 0..6
    const uint32_t s = s7 ^ ((c ^ k) & 0x80808080u);             // sum mod 256
    const uint32_t z = s ^ t4;
    const uint32_t zero = ~(((z & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | z | 0x7F7F7F7Fu);
    const uint32_t ovf = (c & k) | ((c | k) & s7);  // bit 7: carry out of bit 7
    return zero & ~ovf;
}
__device__ __forceinline__ unsigned byte_bits(uint32_t w) {  // bit i = low bit of byte i
    return ((w & 0x01010101u) * 0x01020408u) >> 24;
}
// Bit j of the result is set iff byte j of c + k equals the target (t4 =
// target in all four bytes), for the sixteen bytes of one 16-byte load.
__device__ __forceinline__ unsigned eq_mask8_exact(uint4 c, uint4 k, uint32_t t4) {
    const uint32_t a = byte_marks(c.x, k.x, t4), b = byte_marks(c.y, k.y, t4);
    const uint32_t d = byte_marks(c.z, k.z, t4), e = byte_marks(c.w, k.w, t4);
    return byte_bits(a >> 7) | (byte_bits(b >> 7) << 4) | (byte_bits(d >> 7) << 8) | (byte_bits(e >> 7) << 12);
}
// A first test that most loads settle: nonzero iff some byte of the four
// words may match.  (z - 0x01..) & ~z & 0x80.. is nonzero iff some byte of
// z is zero (exact as an existence test).  F7 (floor(1/eps) <= 125: cbar <=
// 125, keys <= 127): a plain add has no carry between the bytes of real
// columns (padding bytes 0xFF + 0xFF sit above them and never equal a
// target), so z = (c + k) ^ t4.  Otherwise z is formed from the per-byte sum
// mod 256, and a sum that reached 256 can pass; the exact marks settle it.
__device__ __forceinline__ uint32_t zero_byte(uint32_t z) { return (z - 0x01010101u) & ~z & 0x80808080u; }
template <bool F7>
__device__ __forceinline__ uint32_t may_match(uint32_t c, uint32_t k, uint32_t t4) {
    if (F7) return zero_byte((c + k) ^ t4);
    return zero_byte((((c & 0x7F7F7F7Fu) + (k & 0x7F7F7F7Fu)) ^ ((c ^ k) & 0x80808080u)) ^ t4);
}
template <bool F7 = false>
__device__ __forceinline__ unsigned eq_mask8(uint4 c, uint4 k, uint32_t t4) {
    if ((may_match<F7>(c.x, k.x, t4) | may_match<F7>(c.y, k.y, t4) | may_match<F7>(c.z, k.z, t4) |
         may_match<F7>(c.w, k.w, t4)) == 0u)
        return 0u;
    return eq_mask8_exact(c, k, t4);
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
