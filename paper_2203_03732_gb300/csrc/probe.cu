// probe.cu -- pr_probe_latency: the measured floors under one round of the
// phase loop, for a latency roofline.  A round of Sec. 2.2's step (I) with a
// grid-wide round rule cannot take less than one grid barrier plus the
// dependent global round trips it makes (round-start state, row scan,
// proposal atomic); these kernels time each kind of step alone.
#include <cuda_runtime.h>
#include <stdint.h>

#include "prot_internal.cuh"
#include "scan_common.cuh"

namespace prot {
namespace {

constexpr int kProbeThreads = 512;     // the phase kernel's block size
constexpr int kProbeBarriers = 2000;   // barriers timed in a row
constexpr int kProbeChain = 1 << 20;   // 4 MB chain of 32-bit indices (stays in L2)
constexpr int kProbeSteps = 4096;      // dependent loads timed in a row

struct ProbeHead {
    WsHead head;
    unsigned long long slots[4];
    unsigned long long ns[2];  // barrier loop, load chain
    unsigned sink;
    unsigned pad[3];
};

// All CTAs (one per SM) pass kProbeBarriers payload barriers; CTA 0 times them.
__global__ void __launch_bounds__(kProbeThreads, 1)
k_probe_barrier(ProbeHead *ph, long long limit) {
    unsigned gen = 0;
    unsigned long long sum = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) t0 = gtimer();
    for (int i = 0; i < kProbeBarriers; ++i)
        if (!grid_sum_barrier(ph->slots, &ph->head, gen, gridDim.x, limit, 1, sum)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ph->ns[0] = gtimer() - t0;
}

// next[i] = (5 i + 12345) mod 2^20: one cycle through every index (a full
// period linear congruential map: odd increment, multiplier 1 mod 4), and
// consecutive steps land 5 * 4 bytes * i apart, on different lines.
__global__ void k_probe_chain_init(unsigned *next) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kProbeChain; i += gridDim.x * blockDim.x)
        next[i] = (5u * (unsigned)i + 12345u) & (unsigned)(kProbeChain - 1);
}

// One thread follows the chain: every load's address is the last load's
// value, read at L2 (ld.global.cg).
__global__ void k_probe_chase(const unsigned *next, ProbeHead *ph) {
    unsigned i = 0;
    for (int s = 0; s < 64; ++s) asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(i) : "l"(next + i));  // warm
    const unsigned long long t0 = gtimer();
    for (int s = 0; s < kProbeSteps; ++s) asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(i) : "l"(next + i));
    ph->ns[1] = gtimer() - t0;
    ph->sink = i;
}

size_t probe_bytes() { return 256 + (size_t)kProbeChain * sizeof(unsigned); }

}  // namespace
}  // namespace prot

using namespace prot;

extern "C" size_t pr_probe_workspace(void) { return probe_bytes(); }

extern "C" pr_status pr_probe_latency(void *ws, size_t ws_bytes, double *barrier_ns, double *l2_ns, void *stream) {
    if (!barrier_ns || !l2_ns) return fail(PR_ERR_INVALID, "pr_probe_latency: NULL output");
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < probe_bytes())
        return fail(PR_ERR_WORKSPACE, "pr_probe_latency: workspace NULL, not 256-byte aligned or < %zu bytes",
                    probe_bytes());
    cudaStream_t st = (cudaStream_t)stream;
    ProbeHead *ph = (ProbeHead *)ws;
    unsigned *next = (unsigned *)((char *)ws + 256);
    PR_CUDA(cudaMemsetAsync(ph, 0, sizeof(ProbeHead), st));
    const int sms = device_info().sms;
    k_probe_chain_init<<<sms * 4, 256, 0, st>>>(next);
    PR_CUDA(cudaGetLastError());
    long long limit = spin_limit_cycles();
    void *args[] = {(void *)&ph, (void *)&limit};
    PR_CUDA(cudaLaunchCooperativeKernel((const void *)k_probe_barrier, dim3(sms), dim3(kProbeThreads), args, 0, st));
    k_probe_chase<<<1, 1, 0, st>>>(next, ph);
    PR_CUDA(cudaGetLastError());
    ProbeHead h;
    PR_CUDA(cudaMemcpyAsync(&h, ph, sizeof(h), cudaMemcpyDeviceToHost, st));
    PR_CUDA(cudaStreamSynchronize(st));
    if (h.head.err) return fail((pr_status)h.head.err, "pr_probe_latency: a barrier wait ran out");
    *barrier_ns = (double)h.ns[0] / kProbeBarriers;
    *l2_ns = (double)h.ns[1] / kProbeSteps;
    return PR_OK;
}
