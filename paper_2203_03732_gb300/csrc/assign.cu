// assign.cu -- pr_assign: the push-relabel assignment solver on one GB300.
//
// Pipeline (all on the caller's stream, no host round trip inside a solve):
//   k_init      y(b) = 1, y(a) = 0, M empty, B' = all rows        (Sec. 2.2)
//   k_quantise  cbar = floor(c / eps) as uint16, row-major [b][a] (Eq. 1)
//   k_phases    persistent cooperative kernel: all phases, all rounds
//   k_finish    completion + FP64 cost + y(A) output             (Sec. 2.1)
//
// Integer form (units of eps): with k(a) = -y(a) >= 0, an edge is admissible
// (slack 0, Eq. 2 with equality) iff  cbar(b,a) + k(a) == y(b) - 1.  Both
// cbar and k fit 16 bits (Lemma 3.2 bounds |y| by floor(1/eps) + 2), so a
// 16-byte load of eight cbar values is tested against eight k values with
// four 32-bit adds: two 16-bit lanes per word, no carry between them.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "prot_internal.cuh"

namespace prot {
namespace {

constexpr int kThreads = 512;           // threads per CTA of the phase kernel
constexpr int kWarps = kThreads / 32;
constexpr int kUnroll = 8;              // 16-byte loads in flight per lane per chunk
constexpr int kChunk = 32 * 8 * kUnroll;  // cbar elements per warp chunk (4 KiB)
constexpr int kQueue = 1024;            // per-CTA job queue / append buffer capacity
constexpr unsigned long long kEmpty = ~0ull;
constexpr uint16_t kPadCost = 0x7FFF;   // cbar of padding columns
constexpr uint16_t kPadKey = 0x8000;    // k of padding columns: pad sum 0xFFFF never matches

// Control block at the start of the workspace.
struct Ctl {
    WsHead head;
    int nfree[3];        // |B'| lists, ring by phase index
    int nprop[3];        // proposer lists, ring by global step index
    int nwon[2];         // columns won in a phase (prop reset / key update), by phase parity
    int free_at_stop;
    int pad0;
    long long phases;
    long long rounds;
    unsigned long long bytes;
    unsigned long long rows;
};

struct Layout {
    size_t ctl, cb, ka, ptr, prop, freel, propl, wonl, total;
    int ldq;
};

Layout make_layout(int nB, int nA) {
    Layout L;
    Carver c;
    L.ldq = (nA + 7) & ~7;
    L.ctl = c.take<Ctl>(1);
    L.cb = c.take<uint16_t>((size_t)nB * L.ldq);
    L.ka = c.take<uint16_t>(L.ldq);
    L.ptr = c.take<int>(nB);
    L.prop = c.take<unsigned long long>(2 * (size_t)nA);
    L.freel = c.take<int>(3 * (size_t)nB);
    L.propl = c.take<int>(3 * (size_t)nB);
    L.wonl = c.take<int>(2 * (size_t)nB);
    L.total = c.total();
    return L;
}

struct Params {
    Ctl *ctl;
    const uint16_t *cb;
    uint16_t *ka;
    int *y_b;
    int *match_b;
    int *match_a;
    int *ptr;
    unsigned long long *prop;  // [2][nA]
    int *freel;                // [3][nB]
    int *propl;                // [3][nB]
    int *wonl;                 // [2][nB]
    int nB, nA, ldq, T;
    long long phase_cap;
    long long spin_limit;
};

// ---------------------------------------------------------------------------
// k_init
// ---------------------------------------------------------------------------
__global__ void k_init(Params p) {
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int b = t0; b < p.nB; b += stride) {
        p.y_b[b] = 1;
        p.match_b[b] = -1;
        p.freel[b] = b;  // B' of phase 0 = every row
    }
    for (int a = t0; a < p.ldq; a += stride) {
        p.ka[a] = a < p.nA ? 0 : kPadKey;
        if (a < p.nA) {
            p.match_a[a] = -1;
            p.prop[a] = kEmpty;
            p.prop[(size_t)p.nA + a] = kEmpty;
        }
    }
    if (t0 == 0) {
        Ctl *c = p.ctl;
        memset(c, 0, sizeof(Ctl));
        c->head.magic = kWsMagic;
        c->nfree[0] = p.nB;
    }
}

// ---------------------------------------------------------------------------
// k_quantise: cbar = floor(c / eps) with an IEEE FP64 divide (Eq. 1).  One
// thread per 8 consecutive columns of a row; one 16-byte store.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_quantise(const T *__restrict__ C, long long ldc, int nB, int nA, int ldq,
                           double eps, uint16_t *__restrict__ cb, WsHead *head) {
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
                        h[k] = (uint32_t)floor(__ddiv_rn(c, eps));
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

// ---------------------------------------------------------------------------
// Row scan: the lowest column a >= start with cbar(b,a) + k(a) == tgt that no
// earlier round of this phase took.  A warp scans one chunk of kChunk columns
// with kUnroll independent 16-byte loads per lane in flight.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned match_mask(uint4 c, uint4 k, uint32_t tgt2) {
    const uint32_t w0 = (c.x + k.x) ^ tgt2, w1 = (c.y + k.y) ^ tgt2;
    const uint32_t w2 = (c.z + k.z) ^ tgt2, w3 = (c.w + k.w) ^ tgt2;
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

// Returns the column found, or -1.  `ks` points at the phase's key copy
// (shared memory).  Round tags: a column is taken iff its proposal word
// carries a round tag < r.
__device__ __forceinline__ int warp_scan_chunk(const uint16_t *__restrict__ row,
                                               const uint16_t *ks, int c0, int start, int ldq,
                                               uint32_t tgt2,
                                               const unsigned long long *prop, unsigned r,
                                               int lane) {
    uint4 cv[kUnroll], kv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int idx = c0 + u * 256 + lane * 8;
        if (idx < ldq) {
            cv[u] = ld_nc_v4(row + idx);
            kv[u] = *reinterpret_cast<const uint4 *>(ks + idx);
        } else {
            cv[u] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
            kv[u] = make_uint4(0, 0, 0, 0);
        }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int idx = c0 + u * 256 + lane * 8;
        unsigned m = match_mask(cv[u], kv[u], tgt2);
        const int lo = start - idx;
        if (lo > 0) m = lo >= 8 ? 0u : (m & (0xFFu << lo));
        if (__ballot_sync(0xFFFFFFFFu, m != 0) == 0) continue;
        bool found = false;
        int fa = -1;
        for (;;) {
            if (m != 0 && !found) {
                const int a = idx + __ffs(m) - 1;
                const unsigned long long key = ld_relaxed_u64(prop + a);
                if ((unsigned)(key >> 32) < r) {
                    m &= m - 1;  // taken in an earlier round
                } else {
                    found = true;
                    fa = a;
                }
            }
            const unsigned inplay = __ballot_sync(0xFFFFFFFFu, m != 0 || found);
            if (inplay == 0) break;
            const int L = __ffs(inplay) - 1;
            const unsigned fb = __ballot_sync(0xFFFFFFFFu, found);
            if (fb & (1u << L)) return __shfl_sync(0xFFFFFFFFu, fa, L);
        }
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Shared state of one CTA of the phase kernel.
// ---------------------------------------------------------------------------
struct Smem {
    int job_b[kQueue];
    int job_start[kQueue];
    int buf_prop[kQueue];
    int buf_free[kQueue];
    int buf_won[kQueue];
    int n_job, n_prop, n_free, n_won;
    int best[kWarps];
    int base_prop, base_free, base_won;
    unsigned long long bytes;
    unsigned long long rows;
};

__device__ __forceinline__ void flush_lists(Smem &s, const Params &p, int *prop_list,
                                            int *prop_cnt, int *free_list, int *free_cnt,
                                            int *won_list, int *won_cnt) {
    __syncthreads();
    if (threadIdx.x == 0) {
        s.base_prop = s.n_prop ? atomicAdd(prop_cnt, s.n_prop) : 0;
        s.base_free = s.n_free ? atomicAdd(free_cnt, s.n_free) : 0;
        s.base_won = s.n_won ? atomicAdd(won_cnt, s.n_won) : 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < s.n_prop; i += blockDim.x) prop_list[s.base_prop + i] = s.buf_prop[i];
    for (int i = threadIdx.x; i < s.n_free; i += blockDim.x) free_list[s.base_free + i] = s.buf_free[i];
    for (int i = threadIdx.x; i < s.n_won; i += blockDim.x) won_list[s.base_won + i] = s.buf_won[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        s.n_prop = 0;
        s.n_free = 0;
        s.n_won = 0;
        s.n_job = 0;
    }
    __syncthreads();
}

// Scan the queued jobs (row b from column `start`), rows_per_group rows at a
// time, warps_per_row warps per row; then propose or relabel.
__device__ __forceinline__ void run_jobs(Smem &s, const Params &p, const uint16_t *ks,
                                         unsigned long long *prop, unsigned r, int q_phase,
                                         int warps_per_row, int rows_per_group) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nq = s.n_job;
    for (int g0 = 0; g0 < nq; g0 += rows_per_group) {
        const int ng = min(rows_per_group, nq - g0);
        if (threadIdx.x < ng) s.best[threadIdx.x] = 0x7FFFFFFF;
        __syncthreads();
        const int slot = warp / warps_per_row, sub = warp - slot * warps_per_row;
        unsigned long long my_bytes = 0;
        if (slot < ng) {
            const int b = s.job_b[g0 + slot];
            const int start = s.job_start[g0 + slot];
            const int s8 = start & ~7;
            const uint32_t tgt = (uint32_t)(p.y_b[b] - 1);
            const uint32_t tgt2 = tgt | (tgt << 16);
            const uint16_t *row = p.cb + (size_t)b * p.ldq;
            volatile int *vbest = &s.best[slot];
            for (int c0 = s8 + sub * kChunk; c0 < p.ldq; c0 += warps_per_row * kChunk) {
                // warp-uniform early exit: lane 0's view of the row's best so far
                if (c0 >= __shfl_sync(0xFFFFFFFFu, *vbest, 0)) break;
                my_bytes += 2ull * (unsigned long long)min(kChunk, p.ldq - c0);
                const int a = warp_scan_chunk(row, ks, c0, start, p.ldq, tgt2, prop, r, lane);
                if (a >= 0) {
                    if (lane == 0) atomicMin(&s.best[slot], a);
                    break;
                }
            }
        }
        if (lane == 0 && my_bytes) atomicAdd(&s.bytes, my_bytes);
        __syncthreads();
        if (threadIdx.x < ng) {
            const int b = s.job_b[g0 + threadIdx.x];
            const int a = s.best[threadIdx.x];
            if (a != 0x7FFFFFFF) {
                atomicMin(prop + a, ((unsigned long long)r << 32) | (unsigned)b);
                p.ptr[b] = a;
                s.buf_prop[atomicAdd(&s.n_prop, 1)] = b;
            } else {
                p.y_b[b] += 1;  // step (III b): free w.r.t. M' -> relabel
                s.buf_free[atomicAdd(&s.n_free, 1)] = b;
            }
        }
        // the next group's reset of s.best is ordered by the barrier at its top
        __syncthreads();
    }
    if (threadIdx.x == 0) s.rows += (unsigned long long)nq;
}

// ---------------------------------------------------------------------------
// k_phases: every phase of Sec. 2.2 in one cooperative launch.
//
// Phase p (parity q = p & 1) works on B' = freel[p % 3].  Step 1 scans every
// row of B' from column 0.  Step s >= 2 first settles the proposals of step
// s-1: the winner of column a (lowest proposer, atomicMin of (round<<32 | b))
// pushes (a,b) into M, evicts a's old partner into next B' and lowers y(a);
// a loser rescans its row after a.  A row with no admissible untaken column
// relabels (y(b) += 1) and joins next B'.  The phase ends after the first
// step in which nobody proposed; one grid barrier separates steps.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1)
k_phases(Params p, int warps_per_row, int rows_per_group) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ Smem s;
    uint16_t *ks = reinterpret_cast<uint16_t *>(dyn);  // k(a) as of the phase start
    Ctl *ctl = p.ctl;
    WsHead *head = &ctl->head;
    const unsigned G = gridDim.x;
    unsigned gen = 0;

    for (int i = threadIdx.x; i < (p.ldq >> 3); i += blockDim.x)
        reinterpret_cast<uint4 *>(ks)[i] = reinterpret_cast<const uint4 *>(p.ka)[i];
    if (threadIdx.x == 0) {
        s.n_job = s.n_prop = s.n_free = s.n_won = 0;
        s.bytes = 0;
        s.rows = 0;
    }
    __syncthreads();

    long long phase = 0;
    unsigned long long step = 0;
    long long rounds = 0;
    for (;;) {
        const int cur = (int)(phase % 3);
        const int nf = ld_relaxed_s32(&ctl->nfree[cur]);
        if (nf <= p.T) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->free_at_stop = nf;
            break;
        }
        if (phase >= p.phase_cap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                ctl->free_at_stop = nf;
                record_error(head, PR_ERR_NO_CONVERGENCE);
            }
            break;
        }
        const int q = (int)(phase & 1);
        unsigned long long *prop = p.prop + (size_t)q * p.nA;
        unsigned long long *prop_old = p.prop + (size_t)(q ^ 1) * p.nA;
        int *won_list = p.wonl + (size_t)q * p.nB;
        const int *won_old = p.wonl + (size_t)(q ^ 1) * p.nB;
        const int nxt = (int)((phase + 1) % 3);
        int *free_next = p.freel + (size_t)nxt * p.nB;

        // Phase start: columns won in the previous phase have k(a) one higher
        // (step III a); their proposal words are reset for phase p + 1.
        {
            const int nw = phase > 0 ? ld_relaxed_s32(&ctl->nwon[q ^ 1]) : 0;
            for (int i = threadIdx.x; i < nw; i += blockDim.x) ks[won_old[i]] += 1;
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += G * blockDim.x)
                prop_old[won_old[i]] = kEmpty;
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                ctl->nwon[q] = 0;
                ctl->nfree[(phase + 2) % 3] = 0;
            }
            __syncthreads();
        }

        const int *work = p.freel + (size_t)cur * p.nB;
        int nwork = nf;
        unsigned r = 0;
        for (;;) {
            ++r;
            ++step;
            const int si = (int)(step % 3);
            int *prop_list = p.propl + (size_t)si * p.nB;
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->nprop[(step + 1) % 3] = 0;

            // this CTA's items: work[blockIdx.x + k * G], k = 0, 1, ... (cyclic)
            const int my_items = nwork > (int)blockIdx.x ? (nwork - 1 - (int)blockIdx.x) / (int)G + 1 : 0;
            for (int k0 = 0; k0 < my_items; k0 += kQueue) {
                const int cnt = min(kQueue, my_items - k0);
                for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                    const int b = work[blockIdx.x + (size_t)(k0 + i) * G];
                    int start = 0;
                    if (r > 1) {
                        const int a = p.ptr[b];
                        const unsigned long long key = ld_relaxed_u64(prop + a);
                        if (key == (((unsigned long long)(r - 1) << 32) | (unsigned)b)) {
                            // Step (II): push (a,b), evict a's old partner.
                            const int old = p.match_a[a];
                            if (old >= 0) {
                                p.match_b[old] = -1;
                                s.buf_free[atomicAdd(&s.n_free, 1)] = old;
                            }
                            p.match_a[a] = b;
                            p.match_b[b] = a;
                            p.ka[a] += 1;  // step (III a): y(a) -= eps
                            s.buf_won[atomicAdd(&s.n_won, 1)] = a;
                            continue;
                        }
                        start = a + 1;  // lost: resume after a
                    }
                    const int j = atomicAdd(&s.n_job, 1);
                    s.job_b[j] = b;
                    s.job_start[j] = start;
                }
                __syncthreads();
                run_jobs(s, p, ks, prop, r, q, warps_per_row, rows_per_group);
                flush_lists(s, p, prop_list, &ctl->nprop[si], free_next, &ctl->nfree[nxt], won_list,
                            &ctl->nwon[q]);
            }
            if (!grid_barrier(head, gen, G, p.spin_limit)) goto done;
            const int np = ld_relaxed_s32(&ctl->nprop[si]);
            if (np == 0) break;
            ++rounds;
            work = prop_list;
            nwork = np;
        }
        ++phase;
    }
done:
    if (threadIdx.x == 0) {
        if (s.bytes) atomicAdd(&ctl->bytes, s.bytes);
        if (s.rows) atomicAdd(&ctl->rows, s.rows);
        if (blockIdx.x == 0) {
            ctl->phases = phase;
            ctl->rounds = rounds;
        }
    }
}

// ---------------------------------------------------------------------------
// k_finish (one CTA): completion (k-th free row with k-th free column),
// y(A) = -k, and the FP64 matching cost with a fixed-order tree reduction.
// ---------------------------------------------------------------------------
constexpr int kFinThreads = 1024;

__device__ __forceinline__ int block_exclusive_scan(int flag, int *warp_tot, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, flag);
    const int within = __popc(bal & ((1u << lane) - 1));
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
        const int v = lane < (kFinThreads / 32) ? warp_tot[lane] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < (kFinThreads / 32)) warp_tot[lane] = x - v;
        if (lane == 31) *total = x;
    }
    __syncthreads();
    const int r = warp_tot[warp] + within;
    __syncthreads();
    return r;
}

template <class T>
__global__ void __launch_bounds__(kFinThreads)
k_finish(Params p, const T *__restrict__ C, long long ldc, int *free_b, int *free_a,
         int *y_col, double *cost) {
    __shared__ int warp_tot[32];
    __shared__ int total;
    __shared__ double part[kFinThreads];
    if (ld_relaxed_s32(&p.ctl->head.err) != 0) return;
    // ascending free rows
    int nfb = 0;
    for (int base = 0; base < p.nB; base += kFinThreads) {
        const int b = base + threadIdx.x;
        const int f = (b < p.nB && p.match_b[b] < 0) ? 1 : 0;
        const int pos = block_exclusive_scan(f, warp_tot, &total);
        if (f) free_b[nfb + pos] = b;
        nfb += total;
        __syncthreads();
    }
    int nfa = 0;
    for (int base = 0; base < p.nA && nfa < nfb; base += kFinThreads) {
        const int a = base + threadIdx.x;
        const int f = (a < p.nA && p.match_a[a] < 0) ? 1 : 0;
        const int pos = block_exclusive_scan(f, warp_tot, &total);
        if (f && nfa + pos < nfb) free_a[nfa + pos] = a;
        nfa += total;
        __syncthreads();
    }
    for (int k = threadIdx.x; k < nfb; k += kFinThreads) {
        p.match_b[free_b[k]] = free_a[k];
        p.match_a[free_a[k]] = free_b[k];
    }
    for (int a = threadIdx.x; a < p.nA; a += kFinThreads) y_col[a] = -(int)p.ka[a];
    __syncthreads();
    double acc = 0.0;
    for (int b = threadIdx.x; b < p.nB; b += kFinThreads)
        acc = __dadd_rn(acc, (double)C[(long long)b * ldc + p.match_b[b]]);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kFinThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *cost = part[0];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct KernelCfg {
    int grid = 0;
    int dev = -1;
    size_t smem = 0;
};

pr_status launch_phases(const Params &prm, int ldq, cudaStream_t st) {
    const DeviceInfo &di = device_info();
    const size_t smem = (size_t)ldq * sizeof(uint16_t);
    if (smem + sizeof(Smem) > (size_t)di.max_smem_optin)
        return fail(PR_ERR_INVALID, "n_cols too large for the shared-memory key copy");
    PR_CUDA(cudaFuncSetAttribute(k_phases, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phases, kThreads, smem));
    if (per_sm < 1) return fail(PR_ERR_INVALID, "phase kernel does not fit on an SM");
    const int grid = di.sms * per_sm;
    const int chunks = (ldq + kChunk - 1) / kChunk;
    int warps_per_row = chunks < kWarps ? chunks : kWarps;
    int rows_per_group = kWarps / warps_per_row;
    Params pc = prm;
    void *args[] = {(void *)&pc, (void *)&warps_per_row, (void *)&rows_per_group};
    PR_CUDA(cudaLaunchCooperativeKernel((const void *)k_phases, dim3(grid), dim3(kThreads), args,
                                        smem, st));
    return PR_OK;
}

}  // namespace

// Exposed to the other translation units (batched solver reuses the layout).
size_t assign_workspace_bytes(int nB, int nA) { return make_layout(nB, nA).total; }

}  // namespace prot

using namespace prot;

extern "C" size_t pr_assign_workspace(int32_t n_rows, int32_t n_cols) {
    if (n_rows < 1 || n_cols < n_rows || n_cols > (1 << 24)) return 0;
    return make_layout(n_rows, n_cols).total;
}

extern "C" pr_status pr_assign(const void *C, pr_dtype dt, int64_t ldc, int32_t n_rows,
                               int32_t n_cols, double eps, int32_t *row_to_col,
                               int32_t *col_to_row, int32_t *y_row, int32_t *y_col, double *cost,
                               pr_stats *stats, void *ws, size_t ws_bytes, void *stream) {
    if (!C || !row_to_col || !col_to_row || !y_row || !y_col || !cost)
        return fail(PR_ERR_INVALID, "pr_assign: NULL pointer argument");
    if (dt != PR_F32 && dt != PR_F64) return fail(PR_ERR_INVALID, "pr_assign: bad dtype");
    if (n_rows < 1 || n_cols < n_rows || n_cols > (1 << 24))
        return fail(PR_ERR_INVALID, "pr_assign: need 1 <= n_rows <= n_cols <= 2^24");
    if (ldc < n_cols) return fail(PR_ERR_INVALID, "pr_assign: ldc < n_cols");
    if (!(eps > 0.0 && eps < 1.0) || floor(1.0 / eps) > 32766.0)
        return fail(PR_ERR_INVALID, "pr_assign: need 0 < eps < 1 and floor(1/eps) <= 32766");
    const Layout L = make_layout(n_rows, n_cols);
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < L.total)
        return fail(PR_ERR_WORKSPACE, "pr_assign: workspace NULL, not 256-byte aligned or < %zu bytes",
                    L.total);
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;

    Params p;
    p.ctl = (Ctl *)(w + L.ctl);
    p.cb = (const uint16_t *)(w + L.cb);
    p.ka = (uint16_t *)(w + L.ka);
    p.y_b = y_row;
    p.match_b = row_to_col;
    p.match_a = col_to_row;
    p.ptr = (int *)(w + L.ptr);
    p.prop = (unsigned long long *)(w + L.prop);
    p.freel = (int *)(w + L.freel);
    p.propl = (int *)(w + L.propl);
    p.wonl = (int *)(w + L.wonl);
    p.nB = n_rows;
    p.nA = n_cols;
    p.ldq = L.ldq;
    p.T = (int)floor(eps * (double)n_rows);
    const long long K = (long long)floor(1.0 / eps);
    p.phase_cap = ((long long)n_rows * (2 * K + 3)) / (p.T + 1) + 1;
    p.spin_limit = spin_limit_cycles();

    const DeviceInfo &di = device_info();
    k_init<<<di.sms * 2, 256, 0, st>>>(p);
    PR_CUDA(cudaGetLastError());
    const long long groups = (long long)n_rows * (L.ldq >> 3);
    const int qgrid = (int)(groups / 256 + 1 < (long long)di.sms * 8 ? groups / 256 + 1 : di.sms * 8);
    if (dt == PR_F64)
        k_quantise<double><<<qgrid, 256, 0, st>>>((const double *)C, ldc, n_rows, n_cols, L.ldq, eps,
                                                  (uint16_t *)p.cb, &p.ctl->head);
    else
        k_quantise<float><<<qgrid, 256, 0, st>>>((const float *)C, ldc, n_rows, n_cols, L.ldq, eps,
                                                 (uint16_t *)p.cb, &p.ctl->head);
    PR_CUDA(cudaGetLastError());
    cudaEvent_t ev0, ev1;
    kernel_events(&ev0, &ev1);
    if (ev0 && ev1) PR_CUDA(cudaEventRecord(ev0, st));
    pr_status rc = launch_phases(p, L.ldq, st);
    if (rc != PR_OK) return rc;
    if (ev0 && ev1) PR_CUDA(cudaEventRecord(ev1, st));
    // completion lists reuse the proposer-list region (free after the loop)
    int *free_b = p.propl;
    int *free_a = p.propl + n_rows;  // 3*nB ints available; free_a needs <= nB entries
    if (dt == PR_F64)
        k_finish<double><<<1, kFinThreads, 0, st>>>(p, (const double *)C, ldc, free_b, free_a, y_col, cost);
    else
        k_finish<float><<<1, kFinThreads, 0, st>>>(p, (const float *)C, ldc, free_b, free_a, y_col, cost);
    PR_CUDA(cudaGetLastError());

    if (stats) {
        Ctl h;
        PR_CUDA(cudaMemcpyAsync(&h, p.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        PR_CUDA(cudaStreamSynchronize(st));
        stats->phases = h.phases;
        stats->rounds = h.rounds;
        stats->bytes_scanned = (int64_t)h.bytes;
        stats->rows_scanned = (int64_t)h.rows;
        stats->free_at_stop = h.free_at_stop;
        stats->threshold = p.T;
        if (h.head.err != 0)
            return fail((pr_status)h.head.err, "pr_assign: device reported %s",
                        pr_status_string((pr_status)h.head.err));
    }
    return PR_OK;
}
