// prot_internal.cuh -- helpers shared by the library's translation units:
// status plumbing, workspace carving, memory-order primitives and the
// bounded-spin grid barrier used by the persistent phase kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/prot.h"

namespace prot {

// ---------------------------------------------------------------------------
// Host-side status plumbing
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
pr_status fail(pr_status s, const char *fmt, ...);
pr_status cuda_fail(cudaError_t e, const char *what);

#define PR_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return prot::cuda_fail(e_, #call); \
    } while (0)

// Default device-spin budget (clock64 cycles, ~1 s at 2 GHz); the environment
// variable PR_SPIN_LIMIT_CYCLES overrides it (tests use a tiny value to drive
// the time-out path without hanging anything).
long long spin_limit_cycles();

// Events set by pr_set_kernel_events (thread-local; NULL when unset).
void kernel_events(cudaEvent_t *start, cudaEvent_t *stop);

struct DeviceInfo {
    int sms;
    int max_smem_optin;
};
const DeviceInfo &device_info();

// ---------------------------------------------------------------------------
// Workspace carving: every region 256-byte aligned.
// ---------------------------------------------------------------------------
struct Carver {
    size_t off = 0;
    template <class T>
    size_t take(size_t count) {
        size_t o = (off + 255) & ~size_t(255);
        off = o + count * sizeof(T);
        return o;
    }
    size_t total() const { return (off + 255) & ~size_t(255); }
};

// Every workspace starts with this head so pr_ws_status can find the status.
struct WsHead {
    int err;                 // first device error (0 = none)
    int abort;               // set with err: every CTA leaves its loop
    unsigned bar_count;      // grid barrier arrivals
    unsigned bar_gen;        // grid barrier generation
    int magic;               // identifies a workspace written by this library
    int pad[3];
};
constexpr int kWsMagic = 0x70725f31;  // "pr_1"

// ---------------------------------------------------------------------------
// Device memory-order primitives (gpu scope)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int2 ld_relaxed_int2(const int2 *p) {
    int2 v;
    asm volatile("ld.relaxed.gpu.global.v2.s32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint4 ld_nc_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void record_error(WsHead *h, int code) {
    atomicCAS(&h->err, 0, code);
    atomicExch(&h->abort, 1);
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  Thread 0
// of each CTA arrives with a release, the last arrival resets the counter and
// bumps the generation with a release; the others spin with acquire loads for
// at most `limit` clock64 cycles.  On time-out the CTA records PR_ERR_TIMEOUT
// and the abort flag, so every CTA leaves at its next barrier.  Returns false
// when the kernel must stop.
__device__ __forceinline__ bool grid_barrier(WsHead *h, unsigned &gen, unsigned nblocks,
                                             long long limit) {
    __shared__ int s_abort;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned g = gen;
        __threadfence();
        unsigned prev = atomicAdd(&h->bar_count, 1u);
        if (prev == nblocks - 1) {
            h->bar_count = 0;
            __threadfence();
            st_release_u32(&h->bar_gen, g + 1);
        } else {
            long long t0 = clock64();
            while (ld_acquire_u32(&h->bar_gen) == g) {
                if (ld_relaxed_s32(&h->abort)) break;
                if (clock64() - t0 > limit) {
                    record_error(h, PR_ERR_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
        s_abort = ld_relaxed_s32(&h->abort);
    }
    __syncthreads();
    gen += 1;
    return s_abort == 0;
}

// Grid barrier that also sums one value per CTA, rotating over four 64-bit
// slots: barrier h adds (1 | v << 10) to slot h % 4 with a release
// reduction, then polls it (acquire, bounded by `limit` clock64 cycles) until
// the arrival field (bits 0..9, at most 1023 CTAs) reaches the grid size.
// CTA 0 zeroes slot (h + 2) % 4 during barrier h: every CTA read it at
// barrier h - 2, and barrier h + 2 can start only after barrier h + 1, which
// needs CTA 0's arrival.  `sum` receives the sum of the v (54 bits); on
// time-out or abort the call returns false and the kernel must stop.
__device__ __forceinline__ bool grid_sum_barrier(unsigned long long *slots, WsHead *h, unsigned &gen,
                                                 unsigned nblocks, long long limit, unsigned long long v,
                                                 unsigned long long &sum) {
    __shared__ unsigned long long s_pub;
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = gen + 1;
        unsigned long long *slot = slots + (g & 3);
        if (blockIdx.x == 0) slots[(g + 2) & 3] = 0;
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(slot), "l"(1ull | (v << 10)) : "memory");
        unsigned long long w = 0;
        const long long t0 = clock64();
        int ok = 1;
        for (;;) {
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(slot) : "memory");
            if ((w & 1023ull) == (unsigned long long)nblocks) break;
            if (ld_relaxed_s32(&h->abort)) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > limit) {
                record_error(h, PR_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        s_pub = w >> 10;
        s_ok = ok;
    }
    __syncthreads();
    gen += 1;
    sum = s_pub;
    return s_ok != 0;
}

}  // namespace prot
