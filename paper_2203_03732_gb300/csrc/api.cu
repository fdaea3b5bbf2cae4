// api.cu -- status strings, thread-local error text, device queries and the
// workspace status reader shared by every entry point.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>

#include <mutex>

#include "prot_internal.cuh"

namespace prot {

static thread_local char g_err[512] = "no error";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

pr_status fail(pr_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

pr_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return PR_ERR_CUDA;
}

static thread_local cudaEvent_t g_ev_start = nullptr, g_ev_stop = nullptr;

void kernel_events(cudaEvent_t *start, cudaEvent_t *stop) {
    *start = g_ev_start;
    *stop = g_ev_stop;
}

long long spin_limit_cycles() {
    const char *v = getenv("PR_SPIN_LIMIT_CYCLES");
    if (v && *v) {
        long long x = atoll(v);
        if (x > 0) return x;
    }
    return 2000000000LL;
}

const DeviceInfo &device_info() {
    // one entry per device ordinal, filled on first use
    static DeviceInfo infos[64];
    static bool ready[64];
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[dev]) {
        DeviceInfo d{};
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (d.sms <= 0) d.sms = 1;
        infos[dev] = d;
        ready[dev] = true;
    }
    return infos[dev];
}

}  // namespace prot

extern "C" const char *pr_last_error(void) { return prot::g_err; }

extern "C" void pr_set_kernel_events(void *start, void *stop) {
    prot::g_ev_start = (cudaEvent_t)start;
    prot::g_ev_stop = (cudaEvent_t)stop;
}

extern "C" const char *pr_status_string(pr_status s) {
    switch (s) {
        case PR_OK: return "PR_OK";
        case PR_ERR_INVALID: return "PR_ERR_INVALID";
        case PR_ERR_CUDA: return "PR_ERR_CUDA";
        case PR_ERR_TIMEOUT: return "PR_ERR_TIMEOUT";
        case PR_ERR_NO_CONVERGENCE: return "PR_ERR_NO_CONVERGENCE";
        case PR_ERR_WORKSPACE: return "PR_ERR_WORKSPACE";
        case PR_ERR_CAPACITY: return "PR_ERR_CAPACITY";
        case PR_ERR_INTERNAL: return "PR_ERR_INTERNAL";
    }
    return "PR_UNKNOWN";
}

extern "C" pr_status pr_ws_status(const void *ws, void *stream) {
    if (!ws) return prot::fail(PR_ERR_INVALID, "pr_ws_status: NULL workspace");
    prot::WsHead h;
    cudaStream_t st = (cudaStream_t)stream;
    PR_CUDA(cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, st));
    PR_CUDA(cudaStreamSynchronize(st));
    if (h.magic != prot::kWsMagic) return prot::fail(PR_ERR_INVALID, "pr_ws_status: not a solver workspace");
    if (h.err != 0) return prot::fail((pr_status)h.err, "device reported %s", pr_status_string((pr_status)h.err));
    return PR_OK;
}
