// assign.cu -- pr_assign: the push-relabel assignment solver on one GB300.
//
// Pipeline (all on the caller's stream, no host round trip inside a solve):
//   k_init      y(b) = 1, y(a) = 0, M empty                        (Sec. 2.2)
//   k_quantise  cbar = floor(c / eps) exactly, [b][a]: uint8 when
//               floor(1/eps) <= 252, else uint16                   (Eq. 1)
//   k_phases    persistent cooperative kernel: every phase and round
//   k_decode    matching and y(A) out of the per-column words
//   k_finish    completion + FP64 cost                             (Sec. 2.1)
//
// Integer form (units of eps): with k(a) = -y(a) >= 0 an edge is admissible
// (slack 0, Eq. 2 with equality) iff  cbar(b,a) + k(a) == y(b) - 1.  Both
// cbar and k fit 16 bits (Lemma 3.2 bounds |y| by floor(1/eps) + 2), so one
// 16-byte load of eight cbar values meets eight k values in four 32-bit adds
// (two 16-bit lanes per word, no carry between them).  When cbar <= 252 it is
// stored in one byte: the matrix is half the size (100 MB at n = 10,000,
// inside the 126 MB L2, so the later phases' rescans hit L2 instead of HBM),
// and each 16-byte load brings sixteen values, widened to 16-bit lanes.
//
// One 64-bit word per column carries all of step (I) and the matching:
//   word(a) = (R << 32) | (0xFFFFFFFF - b)
// where R is a global round counter (never reset) and b the proposer.  Every
// proposal is an atomicMax, so within a round the lowest b wins, and a later
// phase overwrites an earlier one.  A column is "taken" in the current phase
// iff its tag lies in [first round of the phase, current round).  The word of
// a column last won in an earlier phase names its current partner, so the
// first proposer of a phase learns from atomicMax's return value both that
// it is first and which row step (II) evicts.  Nothing is ever reset.
//
// The duals y(A) must stay fixed within a phase.  Each CTA keeps its own
// shared-memory copy of k(A) and a shared-memory bitmap of the columns taken
// so far in the phase.  The first proposer of a column in round R sets the
// column's bit in round R's global bitmap; at the start of round R + 1 every
// CTA ORs that bitmap into its taken set, and at the start of a new phase it
// adds the whole set to its keys (step III a) and empties it.  Round bitmaps
// rotate over three buffers, so one is cleared while the next is read.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "prot_internal.cuh"
#include "scan_common.cuh"
#include "quantise.cuh"
#include "points.cuh"

namespace prot {
namespace {

constexpr int kThreads = 512;             // threads per CTA of the phase kernel
constexpr int kWarps = kThreads / 32;
constexpr int kUnroll = 3;                // 16-byte loads in flight per lane per chunk (swept: 2..12 at n = 10,000; 3-4 best)
// cbar elements per 16-byte load and per warp chunk (32 lanes x kUnroll
// loads: 1.5 KiB) for the storage type CB
template <class CB> constexpr int kPerLoad = 16 / (int)sizeof(CB);
template <class CB> constexpr int kChunk = 32 * kPerLoad<CB> * kUnroll;
// Byte form: used when floor(1/eps) <= 252.  cbar <= 252, every key
// k(a) <= floor(1/eps) + 2 <= 254 (Lemma 3.2) and every target y(b) - 1 <=
// 253, so a saturating byte add cbar + k that reaches 255 can never equal a
// target, and 255 pads both cbar and keys.
constexpr int kMaxCbar8 = 252;
// floor(1/eps) <= 125: cbar <= 125 and keys <= 127 (Lemma 3.2), so cbar + key
// < 256 and the byte pre-test needs no carry isolation (may_match<true>).
constexpr int kMaxCbar7 = 125;
constexpr int kListSm = 1024;             // proposal-list entries kept in shared memory
constexpr int kKeepMax = 16;              // rows a CTA may keep for its next phase
constexpr int kBatch = 256;               // items turned into scan jobs at a time
constexpr int kMaxGrid = 1023;            // barrier payload field width

// Control block at the start of the workspace.
struct Ctl {
    WsHead head;
    unsigned long long bar_slot[4][2];  // barrier h: arrivals + payload, pool donations
    int pool_cnt[2];                    // pool fill counters, by phase parity
    int free_at_stop;
    int pad0;
    long long phases;
    long long rounds;
    unsigned long long bytes;
    unsigned long long rows;
    unsigned long long cells;  // cost entries the scans examine (start .. answer, or .. row end)
    unsigned maxbits;          // points source: bits of the largest distance (FP32, >= 0)
    int pad1;
    unsigned long long barriers;  // barriers the phase loop passed
    // PR_PROFILE=1: a split of every round (SM clock cycles) into kProfSegs
    // segments: round start (bitmaps, keys), item build, row scans,
    // proposals, donations and the rest, grid barrier; then the item count.
    // prof_own sums CTA 0's values over the rounds, prof_max sums the
    // per-round maximum over CTAs of each segment; prof_rounds counts rounds.
    // The sequential rule (rule_seq.cuh) uses them per phase: segments key
    // update, chains, both; prof_own[3] sums the warps per row.
    unsigned long long prof_own[8];
    unsigned long long prof_max[8];
    unsigned long long prof_slot[2][8];  // per round parity: max over CTAs
    unsigned long long prof_rounds;
    unsigned long long seq_tail;  // PR_RULE_SEQUENTIAL: rows queued so far (rule_seq.cuh)
};
constexpr int kProfSegs = 7;

// Profile clock: the SM's cycle counter (segments are durations within one
// CTA, so counters of different SMs are never compared).
__device__ __forceinline__ unsigned long long ptimer() { return (unsigned long long)clock64(); }

struct Layout {
    size_t ctl, cb, ka, prop, won, pool, lists, ii, total;
    int ldq, won_words;
    size_t list_stride;  // ints per CTA in the list region
};

// Per-CTA overflow storage: two proposal lists of (b, a) pairs (this round,
// previous round), each able to hold every row; the shared pool of free rows
// (two buffers by phase parity).
Layout make_layout(int nB, int nA, int grid) {
    Layout L;
    Carver c;
    L.ldq = (nA + 15) & ~15;  // rows start on 16 bytes in either storage type
    L.ctl = c.take<Ctl>(1);
    L.cb = c.take<uint16_t>((size_t)nB * L.ldq);  // room for the uint16 form
    L.ka = c.take<uint16_t>(L.ldq);
    L.prop = c.take<unsigned long long>((size_t)nA);
    L.won_words = (nA + 31) / 32;
    L.won = c.take<unsigned>(3 * (size_t)L.won_words);
    L.pool = c.take<int2>(2 * (size_t)nB);
    L.list_stride = 8 * (size_t)nB;
    L.lists = c.take<int>((size_t)grid * L.list_stride);
    // PR_RULE_ISRAELI_ITAI's state (rule_ii.cuh): 28 bytes per column, 36 per row
    L.ii = c.take<unsigned long long>((size_t)(2 * nA + nB) + ((size_t)(7 * nB + 3 * nA) + 1) / 2 + 64);
    L.total = c.total();
    return L;
}

struct Params {
    Ctl *ctl;
    const void *cb;  // uint8_t or uint16_t [nB][ldq], as the kernel is instantiated
    uint16_t *ka;
    int *y_b;
    unsigned long long *prop;
    unsigned *won;  // [3][won_words] first proposals of rounds R % 3
    int won_words;
    int2 *pool;  // [2][nB] (b, y(b)) or, for an evicted row, (b, -1 - resume column)
    int *lists;
    size_t list_stride;
    int nB, nA, ldq, T;
    long long phase_cap;
    long long spin_limit;
    int profile;
    int nslots;        // cluster mode: row slots in shared memory (one per scanning warp)
    int slot_bytes;    // bytes per row slot (a whole cbar row, 128-byte multiple)
    int rule = 0;      // step I: 0 lowest-index columns, 1 seeded start columns (PR_RULE_OFFSET),
                       // 2 Israeli-Itai, 3 the sequential greedy by displacement chains
    void *ii = nullptr;  // PR_RULE_ISRAELI_ITAI's state region
};

// PR_RULE_OFFSET: in phase `phase1` (counted from 1) free row b starts its
// scan at column splitmix64(phase1 << 32 | b) mod n_A and goes round the row
// once.  SplitMix64's output function (Steele, Lea and Flood, OOPSLA 2014).
__device__ __forceinline__ int phase_offset(long long phase1, int b, int nA) {
    unsigned long long x = ((unsigned long long)phase1 << 32) | (unsigned)b;
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (int)(x % (unsigned long long)nA);
}

// ---------------------------------------------------------------------------
// k_init
// ---------------------------------------------------------------------------
__global__ void k_init(Params p, int *match_b) {
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int b = t0; b < p.nB; b += stride) {
        p.y_b[b] = 1;
        match_b[b] = -1;
    }
    for (int a = t0; a < p.ldq; a += stride) {
        p.ka[a] = a < p.nA ? 0 : kPadKey;
        if (a < p.nA) p.prop[a] = word_of(0, -1);  // round 0, no partner
    }
    for (int i = t0; i < 3 * p.won_words; i += stride) p.won[i] = 0;
    // every pool slot free (y = 0, see pool_take)
    unsigned long long *pool = reinterpret_cast<unsigned long long *>(p.pool);
    for (long long i = t0; i < 2ll * p.nB; i += stride) pool[i] = 0;
    if (t0 == 0) {
        Ctl *c = p.ctl;
        memset(c, 0, sizeof(Ctl));
        c->head.magic = kWsMagic;
    }
}

// ---------------------------------------------------------------------------
// Row scan against the phase's fixed keys ks (shared memory): the edge (a,b)
// is admissible iff cbar + k(a) == tgt = y(b) - 1.  In the first round of a
// phase nothing is taken; in later rounds a candidate column is skipped when
// its word carries a tag of an earlier round of this phase.
// ---------------------------------------------------------------------------
// Sum of 8 cbar values and their keys (packed 16-bit lanes), from one
// 16-byte load of uint16 cbar.
__device__ __forceinline__ uint4 add_keys(uint4 c, uint4 k) {
    return make_uint4(c.x + k.x, c.y + k.y, c.z + k.z, c.w + k.w);
}

// Lowest candidate column in [c0, c0 + kChunk<CB>) that is >= start and not
// in the phase's taken set tk (shared memory; empty in a phase's first
// round), or -1.  Lane l covers kPerLoad<CB> consecutive columns of each of
// the kUnroll loads, all issued before any is used.
template <class CB, bool F7, bool OFS>
// tgt_in < 0: the row's y(b) is not known yet (an evicted row); lane 0 reads
// it after the row loads are issued, so the two reads overlap.  The target
// used comes back in tgt_out.
// Columns >= stop are not candidates; loads stop at lim (stop rounded up to
// a whole load, <= ldq).
__device__ __forceinline__ int warp_scan_chunk(const CB *__restrict__ row, const CB *ks,
                                               const unsigned *tk, bool check_taken, int c0,
                                               int start, int ldq, int stop, int tgt_in, const int *yb,
                                               int &tgt_out, int lane) {
    constexpr int W = kPerLoad<CB>;
    constexpr unsigned kAll = W == 16 ? 0xFFFFu : 0xFFu;
    uint4 cv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int idx = c0 + u * 32 * W + lane * W;
        cv[u] = idx < ldq ? ld_nc_na_v4(row + idx) : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
    }
    const int tg = tgt_in >= 0 ? tgt_in : __shfl_sync(0xFFFFFFFFu, lane == 0 ? ld_relaxed_s32(yb) - 1 : 0, 0);
    tgt_out = tg;
    const uint32_t tgt = (uint32_t)tg;
    const uint32_t t2 = W == 8 ? (tgt | (tgt << 16)) : tgt * 0x01010101u;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const int idx = c0 + u * 32 * W + lane * W;
        unsigned m = 0;
        if (idx < ldq) {
            const uint4 kv = *reinterpret_cast<const uint4 *>(ks + idx);
            m = W == 8 ? eq_mask(add_keys(cv[u], kv), t2) : eq_mask8<F7>(cv[u], kv, t2);
        }
        const int lo = start - idx;
        if (lo > 0) m &= lo >= W ? 0u : (kAll << lo) & kAll;
        if (OFS) {  // a scan that ends before the row's end (PR_RULE_OFFSET)
            const int hi = stop - idx;
            if (hi < W) m &= hi <= 0 ? 0u : kAll >> (W - hi);
        }
        if (check_taken && m) {
            // the W columns idx .. idx + W - 1 lie in one 32-bit word of the bitmap
            m &= ~(tk[idx >> 5] >> (idx & 31)) & kAll;
        }
        const unsigned any = __ballot_sync(0xFFFFFFFFu, m != 0);
        if (any == 0) continue;
        const int L = __ffs(any) - 1;
        const int a = idx + __ffs(m) - 1;  // meaningful in lane L
        return __shfl_sync(0xFFFFFFFFu, a, L);
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Per-CTA lists: the first kListSm entries in shared memory, the rest in the
// CTA's private region of the workspace.
// ---------------------------------------------------------------------------
struct Smem {
    int2 fl[2][kKeepMax];     // kept rows of this phase / next phase, as pool entries
    int4 ql[2][kListSm];      // (b, a, y(b), origin) proposals of this round / previous round
    int job_b[kBatch];
    int job_start[kBatch];
    int job_stop[kBatch];     // the scan covers columns [start, stop)
    int job_pair[kBatch];     // -1; or the job scanning the row's wrapped part [0, origin); -2 for that job
    int job_tgt[kBatch];
    int job_best[kBatch];
    int2 don[kBatch];         // pool entries given to the pool in this batch
    int best[kWarps];
    int nfl[2], nql[2];
    int njob, ndon, don_base;
    int had_prop, nonfirst, nf_delta, donated;
    unsigned long long bytes;
    unsigned long long rows;
    unsigned long long cells;
    unsigned long long pub, pub2;
    unsigned long long pacc[4];  // profile: build, scan, proposal, tail ns of this round
    unsigned long long cbar[4][2];  // cluster mode: this CTA's copy of the barrier slots
    unsigned long long mbar[kWarps];  // cluster mode: completion of each warp's row copy
    int err;
};

struct Lists {
    int4 *ql[2];  // global overflow of ql
};

__device__ __forceinline__ void ql_push(Smem &s, const Lists &g, int which, int b, int a, int y, int org) {
    const int i = atomicAdd(&s.nql[which], 1);
    if (i < kListSm) s.ql[which][i] = make_int4(b, a, y, org);
    else g.ql[which][i - kListSm] = make_int4(b, a, y, org);
}
__device__ __forceinline__ int4 ql_get(const Smem &s, const Lists &g, int which, int i) {
    return i < kListSm ? s.ql[which][i] : g.ql[which][i - kListSm];
}

// A row of the next phase's B': the CTA keeps up to `keep` of them, the rest
// go to the pool that every CTA draws from at the next phase start.
__device__ __forceinline__ void push_next(Smem &s, int nxt, int keep, int b, int y) {
    const int i = atomicAdd(&s.nfl[nxt], 1);
    if (i < keep) s.fl[nxt][i] = make_int2(b, y);
    else s.don[atomicAdd(&s.ndon, 1)] = make_int2(b, y);
    atomicAdd(&s.nf_delta, 1);
}

// Pool entries: one 64-bit word (b, y), stored and loaded whole.  A real entry
// never has y = 0 (a relabelled row carries y(b) >= 1, an evicted row -2 - a),
// so 0 marks a free slot: k_init clears the pool, and the CTA that takes an
// entry at a phase start clears it again (the slot is written next two phases
// later, behind at least one grid barrier).
__device__ __forceinline__ void pool_put(int2 *pool, long long k, int2 e) {
    const unsigned long long v = ((unsigned long long)(unsigned)e.y << 32) | (unsigned)e.x;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(reinterpret_cast<unsigned long long *>(pool) + k),
                 "l"(v)
                 : "memory");
}
__device__ __forceinline__ unsigned long long pool_raw(const int2 *pool, long long k) {
    return ld_relaxed_u64(reinterpret_cast<const unsigned long long *>(pool) + k);
}
// Takes entry k of this phase's pool given `raw` (an earlier load of it): a
// free slot means the entry was written after its CTA arrived at the phase's
// last barrier (grid_sync_pool) and has not reached L2 yet, so it is loaded
// again, for at most `limit` cycles.  False (and PR_ERR_TIMEOUT) if it never
// arrives.
__device__ __forceinline__ bool pool_take(int2 *pool, long long k, unsigned long long raw, long long limit,
                                          Ctl *ctl, int &b, int &y) {
    if ((unsigned)(raw >> 32) == 0u) {
        const long long t0 = clock64();
        do {
            if (clock64() - t0 > limit) {
                record_error(&ctl->head, PR_ERR_TIMEOUT);
                return false;
            }
            raw = pool_raw(pool, k);
        } while ((unsigned)(raw >> 32) == 0u);
    }
    b = (int)(unsigned)raw;
    y = (int)(raw >> 32);
    pool_put(pool, k, make_int2(0, 0));
    return true;
}

// Grid barrier carrying a payload.  Barrier h adds, for each CTA,
//   1 (arrival) | had_prop << 10 | nonfirst << 20 | nf_delta << 40
// (had_prop, nonfirst in {0,1}; nf_delta < 2^24; at most 1023 CTAs) to word 0
// of slot h % 4 with a release reduction, after adding its pool donations to
// word 1; it then spins (bounded) with acquire loads until the arrival field
// reaches the grid size.  CTA 0 zeroes slot (h + 2) % 4 during round h: every
// CTA read it before arriving at barrier h - 1, and barrier h + 2 reuses it.
// With all_to_pool (no CTA keeps rows: every row of the next phase goes to
// the pool) the pool total equals the summed nf_delta, so word 1 is neither
// added to nor read, which saves a dependent load after every barrier.
// Returns false when the kernel must stop.
__device__ __forceinline__ bool grid_sync(Ctl *ctl, Smem &s, unsigned &gen, unsigned G,
                                          long long limit, unsigned long long mine,
                                          unsigned long long donated, bool all_to_pool) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned h = gen + 1;
        unsigned long long *slot = ctl->bar_slot[h & 3];
        if (blockIdx.x == 0) {
            ctl->bar_slot[(h + 2) & 3][0] = 0;
            ctl->bar_slot[(h + 2) & 3][1] = 0;
        }
        if (donated && !all_to_pool)
            asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(slot + 1), "l"(donated) : "memory");
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(slot), "l"(mine) : "memory");
        unsigned long long v = 0;
        const long long t0 = clock64();
        bool ok = true;
        for (;;) {
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(slot) : "memory");
            if ((v & 1023ull) == (unsigned long long)G) break;
            if (ld_relaxed_s32(&ctl->head.abort)) {
                ok = false;
                break;
            }
            if (clock64() - t0 > limit) {
                record_error(&ctl->head, PR_ERR_TIMEOUT);
                ok = false;
                break;
            }
        }
        const unsigned long long P = (v >> 10) & 1023ull, L = (v >> 20) & 1023ull;
        s.pub = ((P ? 1ull : 0ull) << 31) | ((L ? 1ull : 0ull) << 30) | ((v >> 40) & 0xFFFFFFull);
        s.pub2 = !ok ? 0 : all_to_pool ? ((v >> 40) & 0xFFFFFFull) : ld_relaxed_u64(slot + 1);
        s.err = ok ? 0 : 1;
    }
    __syncthreads();
    gen += 1;
    return s.err == 0;
}

// grid_sync when every next-phase row goes to the pool and a CTA's donations
// of a round fit its shared-memory buffer.  The arrival is an atomic that
// returns the slot's previous value: its nf_delta field (the donations of the
// CTAs that arrived before this one) places this CTA's donations in the pool
// after those of the earlier rounds (pool_base), with no reservation before
// the barrier; the CTA then writes them and waits.  A CTA whose
// arrival completes the count has seen every other arrival (the atomic
// acquires) and does not poll.  Entries written after the last arrival may
// reach L2 after another CTA passed the barrier: pool_take waits for them.
__device__ __forceinline__ bool grid_sync_pool(Ctl *ctl, Smem &s, unsigned &gen, unsigned G, long long limit,
                                               unsigned long long mine, int2 *pool_next, long long pool_base) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned h = gen + 1;
        unsigned long long *slot = ctl->bar_slot[h & 3];
        if (blockIdx.x == 0) {
            ctl->bar_slot[(h + 2) & 3][0] = 0;
            ctl->bar_slot[(h + 2) & 3][1] = 0;
        }
        unsigned long long old;
        asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(slot), "l"(mine) : "memory");
        s.don_base = (int)(pool_base + (long long)((old >> 40) & 0xFFFFFFull));
        s.pub2 = old + mine;  // the slot right after this arrival
    }
    __syncthreads();
    for (int i = threadIdx.x; i < s.ndon; i += blockDim.x) pool_put(pool_next, s.don_base + i, s.don[i]);
    if (threadIdx.x == 0) {
        unsigned long long *slot = ctl->bar_slot[(gen + 1) & 3];
        unsigned long long v = s.pub2;
        bool ok = true;
        if ((v & 1023ull) != (unsigned long long)G) {
            const long long t0 = clock64();
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(slot) : "memory");
                if ((v & 1023ull) == (unsigned long long)G) break;
                if (ld_relaxed_s32(&ctl->head.abort)) {
                    ok = false;
                    break;
                }
                if (clock64() - t0 > limit) {
                    record_error(&ctl->head, PR_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
            }
        }
        const unsigned long long P = (v >> 10) & 1023ull, L = (v >> 20) & 1023ull;
        s.pub = ((P ? 1ull : 0ull) << 31) | ((L ? 1ull : 0ull) << 30) | ((v >> 40) & 0xFFFFFFull);
        s.pub2 = ok ? ((v >> 40) & 0xFFFFFFull) : 0;
        s.err = ok ? 0 : 1;
    }
    __syncthreads();
    gen += 1;
    return s.err == 0;
}

// Cluster form of grid_sync, for a launch that is one thread-block cluster.
// Every CTA holds its own copy of the four slots in shared memory.  At
// barrier h lane r of warp 0 adds the CTA's word 1 and (release, cluster
// scope) word 0 to slot h % 4 of CTA r; thread 0 then polls its own copy
// (bounded, acquire).  Each CTA zeroes its own slot (h + 2) % 4 during round
// h: its last use (barrier h - 2) is over, and no CTA adds to it before
// barrier h + 1 has completed, which needs this CTA's arrival.
__device__ __forceinline__ uint32_t dsmem_addr(const void *p, unsigned rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_barrier_hw() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ bool cluster_sync(Ctl *ctl, Smem &s, unsigned &gen, unsigned G, long long limit,
                                             unsigned long long mine, unsigned long long donated) {
    __syncthreads();
    const unsigned h = gen + 1;
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) {
            s.cbar[(h + 2) & 3][0] = 0;
            s.cbar[(h + 2) & 3][1] = 0;
        }
        if (threadIdx.x < G) {
            const uint32_t r = dsmem_addr(&s.cbar[h & 3][0], threadIdx.x);
            if (donated)
                asm volatile("red.relaxed.cluster.shared::cluster.add.u64 [%0], %1;" ::"r"(r + 8), "l"(donated) : "memory");
            asm volatile("red.release.cluster.shared::cluster.add.u64 [%0], %1;" ::"r"(r), "l"(mine) : "memory");
        }
    }
    if (threadIdx.x == 0) {
        const uint32_t self = dsmem_addr(&s.cbar[h & 3][0], blockIdx.x);
        unsigned long long v = 0;
        const long long t0 = clock64();
        bool ok = true;
        for (;;) {
            asm volatile("ld.acquire.cluster.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(self) : "memory");
            if ((v & 1023ull) == (unsigned long long)G) break;
            if (ld_relaxed_s32(&ctl->head.abort)) {
                ok = false;
                break;
            }
            if (clock64() - t0 > limit) {
                record_error(&ctl->head, PR_ERR_TIMEOUT);
                ok = false;
                break;
            }
        }
        const unsigned long long P = (v >> 10) & 1023ull, L = (v >> 20) & 1023ull;
        s.pub = ((P ? 1ull : 0ull) << 31) | ((L ? 1ull : 0ull) << 30) | ((v >> 40) & 0xFFFFFFull);
        unsigned long long d = 0;
        if (ok) asm volatile("ld.relaxed.cluster.shared::cluster.u64 %0, [%1];" : "=l"(d) : "r"(self + 8) : "memory");
        s.pub2 = d;
        s.err = ok ? 0 : 1;
    }
    __syncthreads();
    gen += 1;
    return s.err == 0;
}

// ---------------------------------------------------------------------------
// Cluster-mode row scan: the row's tail [s_al, ldq) is copied by one bulk
// (TMA) copy into the warp's shared-memory slot, then scanned there.  With one
// slot per warp an SM keeps up to 16 rows (160 KB at n = 10,000) in flight,
// which the 16-byte register loads of the grid form cannot: per SM those
// reach about 64 GB/s from L2, bulk copies about 120 GB/s.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_row_copy(void *dst, const void *src, unsigned bytes, unsigned long long *mbar) {
    // order this warp's earlier reads of the slot (generic proxy) before the
    // copy's writes (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mbar)) : "memory");
}

// Waits (bounded by `limit` cycles) for the phase of parity `parity` of mbar.
__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, unsigned parity, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        unsigned done;
        asm volatile("{ .reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2; selp.u32 %0, 1, 0, q; }"
                     : "=r"(done) : "r"(smem_addr(mbar)), "r"(parity) : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// Lowest candidate column in [start, stop) in the slot holding cbar[s_al ..
// ldq) of one row, ldq here being the end of the copy (the test of
// warp_scan_chunk), or -1.  Four 16-byte shared loads
// per lane are in flight per step.
template <class CB, bool F7, bool OFS>
__device__ __forceinline__ int warp_scan_slot(const unsigned char *slot, const CB *ks, const unsigned *tk,
                                              bool check_taken, int s_al, int start, int ldq, int stop,
                                              uint32_t tgt, int lane) {
    constexpr int W = kPerLoad<CB>;
    constexpr unsigned kAll = W == 16 ? 0xFFFFu : 0xFFu;
    constexpr int kU = 4;
    const uint32_t t2 = W == 8 ? (tgt | (tgt << 16)) : tgt * 0x01010101u;
    for (int e0 = s_al; e0 < ldq; e0 += kU * 32 * W) {
        uint4 cv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int idx = e0 + u * 32 * W + lane * W;
            cv[u] = idx < ldq ? *reinterpret_cast<const uint4 *>(slot + (size_t)(idx - s_al) * sizeof(CB))
                              : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int idx = e0 + u * 32 * W + lane * W;
            unsigned m = 0;
            if (idx < ldq) {
                const uint4 kv = *reinterpret_cast<const uint4 *>(ks + idx);
                m = W == 8 ? eq_mask(add_keys(cv[u], kv), t2) : eq_mask8<F7>(cv[u], kv, t2);
            }
            const int lo = start - idx;
            if (lo > 0) m &= lo >= W ? 0u : (kAll << lo) & kAll;
            if (OFS) {
                const int hi = stop - idx;
                if (hi < W) m &= hi <= 0 ? 0u : kAll >> (W - hi);
            }
            if (check_taken && m) m &= ~(tk[idx >> 5] >> (idx & 31)) & kAll;
            const unsigned any = __ballot_sync(0xFFFFFFFFu, m != 0);
            if (any == 0) continue;
            const int L = __ffs(any) - 1;
            const int a = idx + __ffs(m) - 1;  // meaningful in lane L
            return __shfl_sync(0xFFFFFFFFu, a, L);
        }
    }
    return -1;
}

// A bulk copy's completion wait: long enough for any copy a working GPU
// finishes (about a second), independent of the barrier spin limit.
constexpr long long kCopyWaitCycles = 2000000000ll;

// The queued jobs: the row scans (grid form: rows_per_group rows at a time
// with warps_per_row warps per row; cluster form: one row per warp through
// its slot); then every proposal (atomicMax) or relabel at once; then the
// pool donations.
template <class CB, bool SL, bool F7, bool OFS>
__device__ __forceinline__ void run_jobs(Smem &s, const Lists &g, const Params &p,
                                         const CB *ks, const unsigned *tk, unsigned *won_now,
                                         unsigned R, unsigned Rps, int nxt, int qcur, int keep,
                                         int2 *pool_next, int *pool_cnt, bool defer_don, int warps_per_row,
                                         int rows_per_group, unsigned char *slots, unsigned &mstate,
                                         unsigned long long &cells) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nq = s.njob;
    const unsigned long long tA = p.profile ? ptimer() : 0;
    // More jobs than one register group holds go through the shared-memory
    // slots (up to 16 rows in flight instead of rows_per_group); the choice is
    // this CTA's own.  The slot scan reads every unknown y(b) first (the
    // register scan reads it inside the row scan).
    const bool via_slots = SL && nq > rows_per_group;
    if (via_slots)
        for (int j = threadIdx.x; j < nq; j += blockDim.x)
            if (s.job_tgt[j] < 0) s.job_tgt[j] = ld_relaxed_s32(p.y_b + s.job_b[j]) - 1;
    if (via_slots) {
        // warp w scans jobs w, w + nslots, ... through its own slot
        __syncthreads();
        unsigned long long my_bytes = 0;
        // mstate: bit 0 the parity of the warp's next mbarrier phase; bit 1 a
        // copy whose completion was not seen (after a wait gave up: no more
        // copies, the solve reports PR_ERR_TIMEOUT)
        if (warp < p.nslots) {
            unsigned char *slot = slots + (size_t)warp * p.slot_bytes;
            for (int j = warp; j < nq; j += p.nslots) {
                const int b = s.job_b[j];
                const int start = s.job_start[j];
                const int stop = OFS ? s.job_stop[j] : p.nA;
                const int lim = OFS ? (stop + kPerLoad<CB> - 1) & ~(kPerLoad<CB> - 1) : p.ldq;
                const int s_al = start & ~(kPerLoad<CB> - 1);
                const uint32_t tgt = (uint32_t)s.job_tgt[j];
                int a = -1;
                if (s_al < lim && !(mstate & 2u)) {
                    const unsigned bytes = (unsigned)((lim - s_al) * sizeof(CB));
                    const CB *src = static_cast<const CB *>(p.cb) + (size_t)b * p.ldq + s_al;
                    __syncwarp();
                    if (lane == 0) bulk_row_copy(slot, src, bytes, &s.mbar[warp]);
                    if (mbar_wait(&s.mbar[warp], mstate & 1u, kCopyWaitCycles)) {
                        mstate ^= 1u;
                        my_bytes += bytes;
                        a = warp_scan_slot<CB, F7, OFS>(slot, ks, tk, R > Rps, s_al, start, lim, stop, tgt, lane);
                    } else {
                        mstate |= 2u;
                        if (lane == 0) record_error(&p.ctl->head, PR_ERR_TIMEOUT);
                    }
                }
                if (lane == 0) s.job_best[j] = a >= 0 ? a : 0x7FFFFFFF;
            }
        }
        if (lane == 0 && my_bytes) atomicAdd(&s.bytes, my_bytes);
    } else
    for (int g0 = 0; g0 < nq; g0 += rows_per_group) {
        const int ng = min(rows_per_group, nq - g0);
        if (threadIdx.x < ng) s.best[threadIdx.x] = 0x7FFFFFFF;
        __syncthreads();
        const int slot = warp / warps_per_row, sub = warp - slot * warps_per_row;
        unsigned long long my_bytes = 0;
        if (slot < ng) {
            const int b = s.job_b[g0 + slot];
            const int start = s.job_start[g0 + slot];
            const int stop = OFS ? s.job_stop[g0 + slot] : p.nA;
            const int lim = OFS ? (stop + kPerLoad<CB> - 1) & ~(kPerLoad<CB> - 1) : p.ldq;
            const int s_al = start & ~(kPerLoad<CB> - 1);
            int tgt = s.job_tgt[g0 + slot];
            const CB *row = static_cast<const CB *>(p.cb) + (size_t)b * p.ldq;
            volatile int *vbest = &s.best[slot];
            const bool known = tgt >= 0;
            for (int c0 = s_al + sub * kChunk<CB>; c0 < lim; c0 += warps_per_row * kChunk<CB>) {
                // warp-uniform early exit: lane 0's view of the row's best so far
                if (c0 >= __shfl_sync(0xFFFFFFFFu, *vbest, 0)) break;
                my_bytes += sizeof(CB) * (unsigned long long)min(kChunk<CB>, lim - c0);
                int t_used;
                const int a = warp_scan_chunk<CB, F7, OFS>(row, ks, tk, R > Rps, c0, start, lim, stop, tgt,
                                                      p.y_b + b, t_used, lane);
                tgt = t_used;
                if (a >= 0) {
                    if (lane == 0) atomicMin(&s.best[slot], a);
                    break;
                }
            }
            // the proposal step needs y(b): the first sub-warp stores what it read
            if (!known && sub == 0 && lane == 0)
                s.job_tgt[g0 + slot] = tgt >= 0 ? tgt : ld_relaxed_s32(p.y_b + b) - 1;
        }
        if (lane == 0 && my_bytes) atomicAdd(&s.bytes, my_bytes);
        __syncthreads();
        if (threadIdx.x < ng) s.job_best[g0 + threadIdx.x] = s.best[threadIdx.x];
    }
    __syncthreads();
    const unsigned long long tB = p.profile ? ptimer() : 0;
    for (int j = threadIdx.x; j < nq; j += blockDim.x) {
        const int pair = OFS ? s.job_pair[j] : -1;
        if (pair == -2) continue;  // a row's wrapped part: decided with the row's first job
        const int b = s.job_b[j];
        int a = s.job_best[j];
        const int st = s.job_start[j], sp = OFS ? s.job_stop[j] : p.nA;
        // entries examined: start .. a, or the whole range [start, stop)
        unsigned ex = a != 0x7FFFFFFF ? (unsigned)(a - st + 1) : (st < sp ? (unsigned)(sp - st) : 0u);
        int org = 0;  // PR_RULE_OFFSET: the row's first column in this phase
        if (pair >= 0) {
            const int a2 = s.job_best[pair];
            const int sp2 = s.job_stop[pair];  // the wrapped part is [0, org)
            if (a == 0x7FFFFFFF) {
                a = a2;
                ex += a2 != 0x7FFFFFFF ? (unsigned)(a2 + 1) : (unsigned)sp2;
            }
            org = sp2;
        } else if (OFS) {
            org = sp == p.nA ? 0 : sp;
        }
        cells += ex;
        if (a != 0x7FFFFFFF) {
            const unsigned long long old = atomicMax(p.prop + a, word_of(R, b));
            const unsigned t = tag_of(old);
            if (t < Rps) {
                // first proposal to a in this phase: a is won this round
                // (step III a: y(a) -= eps, applied to the key copies at the
                // next phase) and its old partner is evicted (step II) into
                // the next phase's B'.
                atomicOr(won_now + (a >> 5), 1u << (a & 31));
                // +1 on the 16-bit output key at L2 (no carry leaves the half: k <= 32768)
                atomicAdd(reinterpret_cast<unsigned *>(p.ka + (a & ~1)), (a & 1) ? 0x10000u : 1u);
                const int partner = row_of(old);
                // The evicted row keeps y(b), and every column <= a is above
                // its target for good (its scan that reached a found nothing
                // admissible before a; keys only rise), so its next scan starts
                // at a + 1.  Its y(b) is not known here: the entry carries
                // -1 - (a + 1) instead.
                if (partner >= 0) push_next(s, nxt, keep, partner, -2 - a);
            } else if (t == R) {
                s.nonfirst = 1;
            } else {
                record_error(&p.ctl->head, PR_ERR_INTERNAL);
            }
            ql_push(s, g, qcur, b, a, s.job_tgt[j] + 1, org);
            s.had_prop = 1;
        } else {
            atomicAdd(p.y_b + b, 1);  // step (III b): free w.r.t. M' -> relabel
            push_next(s, nxt, keep, b, s.job_tgt[j] + 2);
        }
    }
    __syncthreads();
    const unsigned long long tC = p.profile ? ptimer() : 0;
    // donations (unless grid_sync_pool places them at the barrier)
    if (!defer_don && s.ndon > 0) {
        if (threadIdx.x == 0) s.don_base = atomicAdd(pool_cnt, s.ndon);
        __syncthreads();
        for (int i = threadIdx.x; i < s.ndon; i += blockDim.x) pool_put(pool_next, s.don_base + i, s.don[i]);
        __syncthreads();
        if (threadIdx.x == 0) {
            s.donated += s.ndon;
            s.ndon = 0;
        }
    }
    if (threadIdx.x == 0) {
        s.rows += (unsigned long long)nq;
        s.njob = 0;
        if (p.profile) {
            s.pacc[1] += tB - tA;
            s.pacc[2] += tC - tB;
            s.pacc[3] += ptimer() - tC;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// k_phases: every phase of Sec. 2.2 in one cooperative launch.
//
// Phase 0 deals rows b = cta + k*G.  Afterwards each CTA keeps up to `keep`
// of the rows it relabelled or evicted; the others go to a pool, dealt out
// cyclically at the next phase start.  Round R of a phase scans the CTA's
// jobs (its rows in the first round; afterwards the rows whose proposal lost,
// resuming after the lost column), then one payload barrier.  If no column
// received two proposals in round R every proposal won and the phase is over;
// otherwise each CTA rereads its proposals' words to find the losers and runs
// round R + 1.
// ---------------------------------------------------------------------------
// Dynamic shared memory of the phase kernel: Smem, the key copy, the taken
// set; in cluster mode then row slots from a 128-byte boundary.
__host__ __device__ inline size_t smem_bytes(int ldq, int key_bytes = 2) {
    return ((sizeof(Smem) + 15) & ~size_t(15)) + (size_t)ldq * key_bytes +
           (size_t)((ldq + 31) / 32) * sizeof(unsigned);
}
__host__ __device__ inline size_t slots_offset(int ldq, int key_bytes) {
    return (smem_bytes(ldq, key_bytes) + 127) & ~size_t(127);
}

// CL: the launch is one thread-block cluster (barriers through distributed
// shared memory) instead of a cooperative grid.  SL: a CTA whose jobs exceed
// one register group scans them from per-warp shared-memory slots filled by
// bulk copies (always with CL).
template <class CB, bool CL, bool SL, bool F7, bool OFS>
__global__ void __launch_bounds__(kThreads, 1)
k_phases(Params p, int warps_per_row, int rows_per_group) {
    extern __shared__ __align__(16) unsigned char dyn[];
    Smem &s = *reinterpret_cast<Smem *>(dyn);
    // key copy k(A) in the storage type of cbar (bytes: padding 0xFF)
    CB *ks = reinterpret_cast<CB *>(dyn + ((sizeof(Smem) + 15) & ~size_t(15)));
    unsigned *tk = reinterpret_cast<unsigned *>(ks + p.ldq);  // taken set of the phase
    // cluster mode: row slots after the taken set, 128-byte aligned
    unsigned char *slots = dyn + slots_offset(p.ldq, (int)sizeof(CB));
    unsigned mstate = 0;  // cluster mode: this warp's copy state (see run_jobs)
    unsigned long long cells = 0;  // this thread's count of examined entries (added up at exit)
    Ctl *ctl = p.ctl;
    const unsigned G = gridDim.x;
    const int cta = blockIdx.x;
    // With at most two rows per register group (long rows) every free row
    // goes to the pool, which deals them out evenly (measured at n = 10,000:
    // 1-3 % faster than keeping one); shorter rows keep up to a group's worth.
    const int keep = rows_per_group > 2 ? min(rows_per_group - 1, kKeepMax) : 0;
    // Every next-phase row goes to the pool and no CTA takes more than kBatch
    // rows in a round (so its donations of a round fit s.don): the barrier
    // places the donations (grid_sync_pool).
    const bool place_at_barrier = !CL && keep == 0 && p.nB <= kBatch * (int)G;
    Lists g;
    int *base = p.lists + (size_t)cta * p.list_stride;
    g.ql[0] = reinterpret_cast<int4 *>(base);
    g.ql[1] = reinterpret_cast<int4 *>(base + 4 * (size_t)p.nB);

    for (int i = threadIdx.x; i < (p.ldq >> 3); i += blockDim.x) {
        const uint4 v = reinterpret_cast<const uint4 *>(p.ka)[i];
        if (sizeof(CB) == 2) {
            reinterpret_cast<uint4 *>(ks)[i] = v;
        } else {  // eight 16-bit keys to bytes; the padding key 0x8000 becomes 0xFF
            uint32_t w[4] = {v.x, v.y, v.z, v.w}, o[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t r = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t k16 = (w[2 * h + q / 2] >> (16 * (q & 1))) & 0xFFFFu;
                    r |= (k16 > 0xFFu ? 0xFFu : k16) << (8 * q);
                }
                o[h] = r;
            }
            reinterpret_cast<uint2 *>(ks)[i] = make_uint2(o[0], o[1]);
        }
    }
    for (int i = threadIdx.x; i < p.won_words; i += blockDim.x) tk[i] = 0;
    if (threadIdx.x == 0) {
        s.nfl[0] = s.nfl[1] = s.nql[0] = s.nql[1] = 0;
        s.njob = s.ndon = 0;
        s.bytes = s.rows = s.cells = 0;
        s.err = 0;
        for (int i = 0; i < 4; ++i) s.cbar[i][0] = s.cbar[i][1] = 0;
        if (SL) {
            for (int w = 0; w < p.nslots; ++w)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s.mbar[w])) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    __syncthreads();
    // Cluster mode: no CTA adds to another's barrier slots before all have
    // started and zeroed them.
    if (CL) cluster_barrier_hw();

    unsigned gen = 0;
    unsigned R = 0;  // global round counter (round tags)
    long long phase = 0, rounds = 0;
    int cur = 0, qcur = 0;
    long long pool_size = 0;  // rows in this phase's pool
    const int first_items = cta < p.nB ? (p.nB - 1 - cta) / (int)G + 1 : 0;
    for (;;) {
        // ---- one phase ----
        const unsigned Rps = R + 1;
        const int pq = (int)(phase & 1);
        int2 *pool_now = p.pool + (size_t)pq * p.nB;
        int2 *pool_next = p.pool + (size_t)(pq ^ 1) * p.nB;
        if (cta == 0 && threadIdx.x == 0) ctl->pool_cnt[pq] = 0;  // for phase + 1's donations
        const int kept = phase == 0 ? first_items : min(s.nfl[cur], keep);
        const int from_pool = (pool_size > cta) ? (int)((pool_size - 1 - cta) / (long long)G) + 1 : 0;
        long long nf_next = 0, pool_next_size = 0;
        bool first_round = true;
        for (;;) {
            ++R;
            const unsigned long long t_r0 = p.profile ? ptimer() : 0;
            unsigned *won_now = p.won + (size_t)(R % 3) * p.won_words;
            if (threadIdx.x == 0) {
                s.pacc[0] = s.pacc[1] = s.pacc[2] = s.pacc[3] = 0;
                s.had_prop = 0;
                s.nonfirst = 0;
                s.nf_delta = 0;
                s.donated = 0;
                s.ndon = 0;
                s.nql[qcur] = 0;
            }
            // items of this round: kept rows + pool share, or last round's proposals
            const int nitems = first_round ? kept + from_pool : s.nql[qcur ^ 1];
            // Issue this thread's first item load and its bitmap-word load
            // before using either, so the two global reads overlap.
            unsigned long long pre_pool = 0;
            unsigned long long pre_word = 0;
            int4 pre_q = make_int4(0, 0, 0, 0);
            const int it0 = threadIdx.x;
            if (it0 < nitems && it0 < kBatch) {
                if (first_round) {
                    if (phase > 0 && it0 >= kept)
                        pre_pool = pool_raw(pool_now, cta + (long long)(it0 - kept) * G);
                } else {
                    pre_q = ql_get(s, g, qcur ^ 1, it0);
                    pre_word = ld_relaxed_u64(p.prop + pre_q.y);
                }
            }
            const unsigned *wprev = p.won + (size_t)((R + 2) % 3) * p.won_words;
            unsigned pre_m = 0;
            if (R > 1 && threadIdx.x < p.won_words) pre_m = ld_relaxed_u32(wprev + threadIdx.x);
            if (R > 1) {
                // first proposals of round R - 1 join the taken set; a new
                // phase first moves the finished phase's set into the keys
                for (int i = threadIdx.x; i < p.won_words; i += blockDim.x) {
                    unsigned m = i == (int)threadIdx.x ? pre_m : ld_relaxed_u32(wprev + i);
                    if (first_round) {
                        m |= tk[i];
                        tk[i] = 0;
                        while (m) {
                            ks[i * 32 + __ffs(m) - 1] += (CB)1;
                            m &= m - 1;
                        }
                    } else {
                        tk[i] |= m;
                    }
                }
                // round R - 2's bitmap has been read by every CTA: clear it for R + 1
                unsigned *wold = p.won + (size_t)((R + 1) % 3) * p.won_words;
                for (int i = cta * blockDim.x + threadIdx.x; i < p.won_words; i += G * blockDim.x)
                    wold[i] = 0;
            }
            __syncthreads();
            const unsigned long long t_r1 = p.profile ? ptimer() : 0;
            unsigned long long t_mark = t_r1;
            // PR_RULE_OFFSET turns a row into up to two jobs: half as many per batch
            const int per_batch = OFS ? kBatch / 2 : kBatch;
            for (int i0 = 0; i0 < nitems; i0 += per_batch) {
                const int cnt = min(per_batch, nitems - i0);
                for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                    const int it = i0 + i;
                    const bool pre = i0 == 0 && i == (int)threadIdx.x;  // loaded above
                    // the row's scan covers [start, stop), then [0, wrap) if wrap > 0
                    int b, y = -1, start = 0, stop = p.nA, wrap = 0;
                    if (first_round) {
                        if (phase == 0) {
                            b = cta + it * (int)G;
                            y = 1;
                        } else if (it < kept) {
                            const int2 e = s.fl[cur][it];
                            b = e.x;
                            y = e.y;
                        } else {
                            const long long k = cta + (long long)(it - kept) * G;
                            if (!pool_take(pool_now, k, pre ? pre_pool : pool_raw(pool_now, k), p.spin_limit, ctl, b, y))
                                continue;  // PR_ERR_TIMEOUT: the kernel stops at the next barrier
                        }
                        if (y < 0) {  // an evicted row: y(b) unknown, resume point -1 - y
                            start = -1 - y;
                            y = -1;
                        }
                        if (OFS) {  // once round the row from its seeded first column
                            start = phase_offset(phase + 1, b, p.nA);
                            wrap = start;
                        }
                    } else {
                        const int4 q = pre ? pre_q : ql_get(s, g, qcur ^ 1, it);
                        const unsigned long long w = pre ? pre_word : ld_relaxed_u64(p.prop + q.y);
                        b = q.x;
                        if (row_of(w) == b) continue;  // won: matched, leaves B'
                        start = q.y + 1;               // lost: resume after a
                        y = q.z;
                        // PR_RULE_OFFSET (first column q.w): before the wrap the rest
                        // of the row and then [0, q.w); after it, up to q.w
                        if (OFS && q.w > 0) {
                            if (q.y >= q.w) wrap = q.w;
                            else stop = q.w;
                        }
                    }
                    const int tg = y >= 0 ? y - 1 : -1;
                    const int nj = wrap > 0 ? 2 : 1;
                    const int j = atomicAdd(&s.njob, nj);
                    s.job_b[j] = b;
                    s.job_start[j] = start;
                    s.job_tgt[j] = tg;
                    if (OFS) {
                        s.job_stop[j] = stop;
                        s.job_pair[j] = nj == 2 ? j + 1 : -1;
                    }
                    if (OFS && nj == 2) {
                        s.job_b[j + 1] = b;
                        s.job_start[j + 1] = 0;
                        s.job_stop[j + 1] = wrap;
                        s.job_tgt[j + 1] = tg;
                        s.job_pair[j + 1] = -2;
                    }
                }
                __syncthreads();
                if (p.profile && threadIdx.x == 0) s.pacc[0] += ptimer() - t_mark;
                run_jobs<CB, SL, F7, OFS>(s, g, p, ks, tk, won_now, R, Rps, cur ^ 1, qcur, keep, pool_next,
                                          &ctl->pool_cnt[pq ^ 1], place_at_barrier, warps_per_row, rows_per_group,
                                          slots, mstate, cells);
                if (p.profile) t_mark = ptimer();
            }
            const unsigned long long mine = 1ull | ((unsigned long long)s.had_prop << 10) |
                                            ((unsigned long long)s.nonfirst << 20) |
                                            ((unsigned long long)s.nf_delta << 40);
            const unsigned long long t_r2 = p.profile ? ptimer() : 0;
            unsigned long long seg[kProfSegs] = {};
            if (p.profile && threadIdx.x == 0) {
                seg[0] = t_r1 - t_r0;
                seg[1] = s.pacc[0];
                seg[2] = s.pacc[1];
                seg[3] = s.pacc[2];
                seg[4] = s.pacc[3] + (t_r2 - t_mark);
                seg[6] = (unsigned long long)nitems;
                for (int k = 0; k < kProfSegs; ++k)
                    if (k != 5) atomicMax(&ctl->prof_slot[R & 1][k], seg[k]);
                if (cta == 0) {
                    // read after round R - 1; written again (the barrier
                    // segment of round R) only after this barrier
                    for (int k = 0; k < kProfSegs; ++k) ctl->prof_slot[(R + 1) & 1][k] = 0;
                }
            }
            const bool synced =
                CL ? cluster_sync(ctl, s, gen, G, p.spin_limit, mine, (unsigned long long)s.donated)
                : place_at_barrier
                    ? grid_sync_pool(ctl, s, gen, G, p.spin_limit, mine, pool_next, pool_next_size)
                    : grid_sync(ctl, s, gen, G, p.spin_limit, mine, (unsigned long long)s.donated, keep == 0);
            if (!synced) goto done;
            if (p.profile && threadIdx.x == 0) {
                seg[5] = ptimer() - t_r2;
                // the barrier segment of round R goes to the next round's slot
                atomicMax(&ctl->prof_slot[(R + 1) & 1][5], seg[5]);
                if (cta == 0) {
                    for (int k = 0; k < kProfSegs; ++k) {
                        ctl->prof_own[k] += seg[k];
                        ctl->prof_max[k] += ctl->prof_slot[R & 1][k];
                    }
                    ctl->prof_rounds += 1;
                }
            }
            const unsigned long long pub = s.pub;
            if ((pub >> 31) & 1ull) ++rounds;
            nf_next += (long long)(pub & 0x3FFFFFFFull);
            pool_next_size += (long long)s.pub2;
            first_round = false;
            qcur ^= 1;
            if (!((pub >> 30) & 1ull)) break;  // no contested column: phase over
        }
        ++phase;
        if (threadIdx.x == 0) s.nfl[cur] = 0;
        cur ^= 1;
        pool_size = pool_next_size;
        if (nf_next <= p.T) {
            if (cta == 0 && threadIdx.x == 0) ctl->free_at_stop = (int)nf_next;
            break;
        }
        if (phase >= p.phase_cap) {
            if (cta == 0 && threadIdx.x == 0) {
                ctl->free_at_stop = (int)nf_next;
                record_error(&ctl->head, PR_ERR_NO_CONVERGENCE);
            }
            break;
        }
    }
done:
    if (cells) atomicAdd(&s.cells, cells);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s.bytes) atomicAdd(&ctl->bytes, s.bytes);
        if (s.rows) atomicAdd(&ctl->rows, s.rows);
        if (s.cells) atomicAdd(&ctl->cells, s.cells);
        if (cta == 0) {
            ctl->phases = phase;
            ctl->rounds = rounds;
            ctl->barriers = gen;
        }
    }
    // A copy whose wait gave up gets one more bounded wait: the CTA must not
    // exit while it may still write the slot.
    if (SL && (mstate & 2u)) mbar_wait(&s.mbar[threadIdx.x >> 5], mstate & 1u, kCopyWaitCycles);
    // Cluster mode: a CTA's shared memory must outlive every add another CTA
    // makes to it.  Every CTA gets here: the loop ends on the same shared
    // decision everywhere, or on a bounded wait that gave up.
    if (CL) {
        __syncthreads();
        cluster_barrier_hw();
    }
}

#include "rule_ii.cuh"
#include "rule_seq.cuh"

// ---------------------------------------------------------------------------
// k_decode: the matching is the per-column words' rows; y(A) = -k.
// ---------------------------------------------------------------------------
__global__ void k_decode(Params p, int *match_b, int *match_a, int *y_col) {
    if (ld_relaxed_s32(&p.ctl->head.err) != 0) return;
    const int stride = gridDim.x * blockDim.x;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < p.nA; a += stride) {
        const unsigned long long w = p.prop[a];
        const int b = tag_of(w) > 0 ? row_of(w) : -1;
        match_a[a] = b;
        if (b >= 0) match_b[b] = a;
        y_col[a] = -(int)p.ka[a];
    }
}

// ---------------------------------------------------------------------------
// k_finish (one CTA): completion (k-th free row with k-th free column) and the
// FP64 matching cost with a fixed-order tree reduction.
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

// The matched costs k_finish adds up: from the input matrix, or the FP64
// distance of the matched points (input units).
template <class T>
struct MatrixCost {
    const T *C;
    long long ldc;
    __device__ double operator()(int b, int a) const { return (double)C[(long long)b * ldc + a]; }
};
struct PointsCost {
    const float *XA, *XB;
    int dim, squared;
    __device__ double operator()(int b, int a) const {
        return dist_f64(XB + (long long)b * dim, XA + (long long)a * dim, dim, squared);
    }
};

template <class Src>
__global__ void __launch_bounds__(kFinThreads)
k_finish(Params p, Src src, int *match_b, int *match_a, int *free_b, int *free_a, double *cost) {
    __shared__ int warp_tot[32];
    __shared__ int total;
    __shared__ double part[kFinThreads];
    if (ld_relaxed_s32(&p.ctl->head.err) != 0) return;
    int nfb = 0;
    for (int base = 0; base < p.nB; base += kFinThreads) {
        const int b = base + threadIdx.x;
        const int f = (b < p.nB && match_b[b] < 0) ? 1 : 0;
        const int pos = block_exclusive_scan(f, warp_tot, &total);
        if (f) free_b[nfb + pos] = b;
        nfb += total;
        __syncthreads();
    }
    int nfa = 0;
    for (int base = 0; base < p.nA && nfa < nfb; base += kFinThreads) {
        const int a = base + threadIdx.x;
        const int f = (a < p.nA && match_a[a] < 0) ? 1 : 0;
        const int pos = block_exclusive_scan(f, warp_tot, &total);
        if (f && nfa + pos < nfb) free_a[nfa + pos] = a;
        nfa += total;
        __syncthreads();
    }
    for (int k = threadIdx.x; k < nfb; k += kFinThreads) {
        match_b[free_b[k]] = free_a[k];
        match_a[free_a[k]] = free_b[k];
    }
    __syncthreads();
    double acc = 0.0;
    for (int b = threadIdx.x; b < p.nB; b += kFinThreads)
        acc = __dadd_rn(acc, src(b, match_b[b]));
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kFinThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *cost = part[0];
}

// ---------------------------------------------------------------------------
// Costs from points (points.cuh), over the same (row, group of 8 columns)
// grid stride as k_quantise: first the largest distance, then Eq. (1) on
// c = RN32(d / max d), exactly as for a stored FP32 cost.  The largest
// distance is taken over the squared sums: the IEEE square root is correctly
// rounded and non-decreasing, so the root of the largest sum is the largest
// root.
// ---------------------------------------------------------------------------
// The squared sums of row point xb against the 8 column points a0 .. a0+7
// (entries past n_A are left alone).  D > 0: dim == D with XA 16-byte
// aligned, so a group of 8 points is whole 16-byte loads (2 * D of them);
// D == 0: any dim, one coordinate at a time.  Same IEEE operations in the
// same order either way (dist_f32).
template <int D>
__device__ __forceinline__ void sq_group8(const float *__restrict__ XA, const float *__restrict__ xb, int dim,
                                          int a0, int nA, float (&d)[8]) {
    if (D > 0 && a0 + 8 <= nA) {
        float x[8 * (D > 0 ? D : 1)];
        const float4 *v = reinterpret_cast<const float4 *>(XA + (long long)a0 * D);
#pragma unroll
        for (int q = 0; q < 2 * D; ++q) {
            const float4 t = __ldg(v + q);
            x[4 * q] = t.x;
            x[4 * q + 1] = t.y;
            x[4 * q + 2] = t.z;
            x[4 * q + 3] = t.w;
        }
        float xbk[D > 0 ? D : 1];
#pragma unroll
        for (int k = 0; k < D; ++k) xbk[k] = xb[k];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float t = __fsub_rn(xbk[k], x[j * D + k]);
                const float sq = __fmul_rn(t, t);
                acc = k == 0 ? sq : __fadd_rn(acc, sq);
            }
            d[j] = acc;
        }
        return;
    }
    for (int j = 0; j < 8; ++j)
        if (a0 + j < nA) d[j] = dist_f32(xb, XA + (long long)(a0 + j) * dim, dim, 1);
}

template <int D>
__global__ void k_points_max(const float *__restrict__ XA, const float *__restrict__ XB, int dim,
                             int nB, int nA, int ldq, unsigned *maxbits) {
    const long long groups = (long long)nB * (ldq >> 3);
    float m = 0.0f;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
         g += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(g / (ldq >> 3));
        const int a0 = (int)(g - (long long)b * (ldq >> 3)) << 3;
        float d[8];
        sq_group8<D>(XA, XB + (long long)b * dim, dim, a0, nA, d);
        for (int j = 0; j < 8 && a0 + j < nA; ++j) m = fmaxf(m, d[j]);
    }
    // non-negative floats order like their bit patterns (NaN is dropped by fmaxf)
    const unsigned mx = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(m));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(maxbits, mx);
}

template <class CB, int D>
__global__ void k_points_quant(const float *__restrict__ XA, const float *__restrict__ XB, int dim, int squared,
                               int nB, int nA, int ldq, const unsigned *__restrict__ maxbits, EpsSplit e,
                               CB *__restrict__ cb, WsHead *head) {
    constexpr uint32_t kPad = sizeof(CB) == 1 ? 0xFFu : (uint32_t)kPadCost;
    const long long groups = (long long)nB * (ldq >> 3);
    const float M = squared ? __uint_as_float(*maxbits) : __fsqrt_rn(__uint_as_float(*maxbits));
    bool bad = false;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
         g += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(g / (ldq >> 3));
        const int a0 = (int)(g - (long long)b * (ldq >> 3)) << 3;
        float sq[8];
        sq_group8<D>(XA, XB + (long long)b * dim, dim, a0, nA, sq);
        uint32_t h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int a = a0 + j;
            if (a < nA) {
                const float d = squared ? sq[j] : __fsqrt_rn(sq[j]);
                if (!(d >= 0.0f && d <= M)) {  // NaN or infinite coordinates
                    bad = true;
                    h[j] = 0;
                    continue;
                }
                const float c = M > 0.0f ? __fdiv_rn(d, M) : 0.0f;
                h[j] = quantise_fbits(__float_as_uint(c), e);
                if (h[j] == 0xFFFFFFFFu) {  // c not in [0, 1]: an infinite largest distance
                    bad = true;
                    h[j] = 0;
                }
            } else {
                h[j] = kPad;
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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct PhaseCfg {
    int grid = 0;     // grid mode: one CTA per SM (cooperative launch)
    int cluster = 0;  // cluster mode: CTAs in the one cluster (0: not available)
    size_t smem = 0;
};

template <class CB, bool CL, bool SL, bool F7, bool OFS = false>
pr_status set_phase_attrs(size_t smem) {
    PR_CUDA(cudaFuncSetAttribute(k_phases<CB, CL, SL, F7, OFS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (CL) PR_CUDA(cudaFuncSetAttribute(k_phases<CB, CL, SL, F7, OFS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return PR_OK;
}

// The phase kernel for the storage type (cb8: bytes), the form (cl: one
// cluster, sl: row slots), the byte pre-test (f7: floor(1/eps) <= 125) and
// the step I rule (ofs: PR_RULE_OFFSET).
template <bool OFS>
const void *phase_kernel_of(bool cb8, bool cl, bool sl, bool f7) {
    if (!cb8)
        return cl ? (const void *)k_phases<uint16_t, true, true, false, OFS>
                  : sl ? (const void *)k_phases<uint16_t, false, true, false, OFS>
                       : (const void *)k_phases<uint16_t, false, false, false, OFS>;
    if (f7)
        return cl ? (const void *)k_phases<uint8_t, true, true, true, OFS>
                  : sl ? (const void *)k_phases<uint8_t, false, true, true, OFS>
                       : (const void *)k_phases<uint8_t, false, false, true, OFS>;
    return cl ? (const void *)k_phases<uint8_t, true, true, false, OFS>
              : sl ? (const void *)k_phases<uint8_t, false, true, false, OFS>
                   : (const void *)k_phases<uint8_t, false, false, false, OFS>;
}
const void *phase_kernel(bool cb8, bool cl, bool sl, bool f7, bool ofs) {
    return ofs ? phase_kernel_of<true>(cb8, cl, sl, f7) : phase_kernel_of<false>(cb8, cl, sl, f7);
}

// Largest cluster (16, else 8) of k_phases<CB, true, true, false, false> the device can hold, or 0.
template <class CB>
int max_phase_cluster(size_t smem) {
    for (int cs : {16, 8}) {
        cudaLaunchConfig_t c = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        c.gridDim = dim3(cs);
        c.blockDim = dim3(kThreads);
        c.dynamicSmemBytes = smem;
        c.attrs = at;
        c.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, (const void *)k_phases<CB, true, true, false, false>, &c) == cudaSuccess && n >= 1)
            return cs;
        cudaGetLastError();  // clear a refusal of this size
    }
    return 0;
}



pr_status phase_cfg(PhaseCfg &cfg) {
    static int cached_dev = -1;
    static PhaseCfg cached;
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    if (dev == cached_dev) {
        cfg = cached;
        return PR_OK;
    }
    const DeviceInfo &di = device_info();
    const size_t smem = (size_t)di.max_smem_optin;  // Smem + the key copy; see smem_bytes()
    pr_status rc = set_phase_attrs<uint8_t, false, false, false>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint16_t, false, false, false>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, false, true, false>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint16_t, false, true, false>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, true, true, false>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint16_t, true, true, false>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, false, false, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, false, true, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, true, true, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint16_t, false, false, false, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint16_t, false, true, false, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint16_t, true, true, false, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, false, false, false, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, false, true, false, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, true, true, false, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, false, false, true, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, false, true, true, true>(smem);
    if (rc == PR_OK) rc = set_phase_attrs<uint8_t, true, true, true, true>(smem);
    if (rc != PR_OK) return rc;
    int per_sm = 0, per_sm16 = 0;
    PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phases<uint8_t, false, false, false, false>, kThreads, smem));
    PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm16, k_phases<uint16_t, false, false, false, false>, kThreads, smem));
    if (per_sm16 < per_sm) per_sm = per_sm16;
    if (per_sm < 1) return fail(PR_ERR_INVALID, "phase kernel does not fit on an SM");
    int grid = di.sms * per_sm;
    if (grid > kMaxGrid) grid = kMaxGrid;
    cfg.grid = grid;
    const int c8 = max_phase_cluster<uint8_t>(smem), c16 = max_phase_cluster<uint16_t>(smem);
    cfg.cluster = c8 < c16 ? c8 : c16;
    cfg.smem = smem;  // the most a launch may ask for; each launch asks smem_bytes(ldq)
    cached = cfg;
    cached_dev = dev;
    return PR_OK;
}

// The phase loop runs in one thread-block cluster (barriers through
// distributed shared memory, about a third of a grid barrier's latency) or
// on the whole grid (one CTA per SM, barriers through L2).  PR_PHASE_MODE =
// "grid" or "cluster" forces one; otherwise the cluster runs problems of up
// to kClusterMaxRows rows with floor(1/eps) > kClusterMinK.
// Cluster mode also needs at least kMinSlots row slots next to the keys.
constexpr int kMinSlots = 4;

// Measured on GB300 (eps = 0.01): the cluster is ahead up to a few thousand
// rows (n = 2000: 15 %, n = 4000: 6 %); at n = 10,000 the 16 SMs' scan
// throughput falls behind the whole grid's (37 % slower).
constexpr int kClusterMaxRows = 4096;
// ... and only when floor(1/eps) > 20: at larger eps a solve is one phase of
// many rounds with many rows, where the whole grid's scans win (eps = 0.1:
// n = 1000 0.152 vs 0.169 ms, n = 3000 0.333 vs 0.505 ms, grid vs cluster;
// eps = 0.01: 8.24 vs 7.42 ms and 1.97 vs 1.99 ms).
constexpr long long kClusterMinK = 20;

bool use_cluster(const PhaseCfg &cfg, int nslots, int n_rows, long long K) {
    if (cfg.cluster < 1 || nslots < kMinSlots) return false;
    const char *m = getenv("PR_PHASE_MODE");
    if (m && strcmp(m, "grid") == 0) return false;
    if (m && strcmp(m, "cluster") == 0) return true;
    return n_rows <= kClusterMaxRows && K > kClusterMinK;
}

// Row scans of the grid form: a CTA with more jobs than one register group
// sends them through shared-memory slots (measured at n = 10,000: eps = 0.1,
// about 30 rows per CTA per round, 1.00 ms instead of 2.33 ms for the phase
// loop; at eps = 0.01 the rounds hold 4 or 5 rows and stay on registers).
// PR_SCAN=regs keeps every scan on registers.
bool use_slots_in_grid(int nslots) {
    if (nslots < kMinSlots) return false;
    const char *m = getenv("PR_SCAN");
    return !(m && strcmp(m, "regs") == 0);
}

// Where the costs come from: a matrix (C, dt, ldc) or two point sets (XA the
// columns, XB the rows, `dim` FP32 coordinates each).  With `host` set, the
// matrix is in host memory and C is the device buffer it is copied into.
struct CostSource {
    const void *C = nullptr;
    const void *host = nullptr;
    pr_dtype dt = PR_F64;
    int64_t ldc = 0;
    const float *XA = nullptr, *XB = nullptr;
    int dim = 0, squared = 0;
    bool points = false;
};

// The two passes that form the rounded costs from points.
template <int D>
void launch_points(const CostSource &src, int n_rows, int n_cols, const Params &p, const EpsSplit &e, bool cb8,
                   void *cbw, int qgrid, cudaStream_t st) {
    k_points_max<D><<<qgrid, 256, 0, st>>>(src.XA, src.XB, src.dim, n_rows, n_cols, p.ldq, &p.ctl->maxbits);
    if (cb8)
        k_points_quant<uint8_t, D><<<qgrid, 256, 0, st>>>(src.XA, src.XB, src.dim, src.squared, n_rows, n_cols,
                                                          p.ldq, &p.ctl->maxbits, e, (uint8_t *)cbw, &p.ctl->head);
    else
        k_points_quant<uint16_t, D><<<qgrid, 256, 0, st>>>(src.XA, src.XB, src.dim, src.squared, n_rows, n_cols,
                                                           p.ldq, &p.ctl->maxbits, e, (uint16_t *)cbw, &p.ctl->head);
}

// pr_assign_staged's copy stream and chunk events, one set per device, made
// on first use and kept.  A solve enqueues its whole copy and rounding
// sequence under g_stage_mu, so no other solve re-records an event between
// its record and the wait that pairs with it.
constexpr size_t kStageBytes = (size_t)32 << 20;  // host bytes per chunk
constexpr int kStageMaxChunks = 64;
constexpr int kStageMaxDevices = 64;
struct StageRes {
    cudaStream_t copy = nullptr;
    cudaEvent_t start = nullptr;
    cudaEvent_t done[kStageMaxChunks] = {};
};
std::mutex g_stage_mu;
StageRes g_stage[kStageMaxDevices];

template <class T, class CB>
void launch_quantise_rows(const CostSource &src, const Params &p, int r0, int rows, double eps, int sms,
                          cudaStream_t st) {
    const long long groups = (long long)rows * (p.ldq >> 3);
    const long long want = groups / 256 + 1;
    const int grid = (int)(want < (long long)sms * 16 ? want : (long long)sms * 16);
    launch_quantise<T, CB>((const T *)src.C + (size_t)r0 * src.ldc, src.ldc, rows, p.nA, p.ldq, eps,
                           (CB *)const_cast<void *>(p.cb) + (size_t)r0 * p.ldq, &p.ctl->head, grid, st);
}

// Eq. 1 for a host matrix: its rows go to the device buffer src.C in chunks
// of about kStageBytes on the copy stream, and each chunk is rounded on `st`
// as soon as it has arrived, while the next chunk is being copied.  The copy
// stream first waits for the work already on `st`, so a buffer that earlier
// work on `st` still reads is not overwritten early.
pr_status stage_and_round(const CostSource &src, const Params &p, double eps, bool cb8, cudaStream_t st) {
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStageMaxDevices) return fail(PR_ERR_INVALID, "pr_assign_staged: device %d", dev);
    std::lock_guard<std::mutex> lock(g_stage_mu);
    StageRes &R = g_stage[dev];
    if (!R.copy) {
        PR_CUDA(cudaStreamCreateWithFlags(&R.copy, cudaStreamNonBlocking));
        PR_CUDA(cudaEventCreateWithFlags(&R.start, cudaEventDisableTiming));
        for (int k = 0; k < kStageMaxChunks; ++k)
            PR_CUDA(cudaEventCreateWithFlags(&R.done[k], cudaEventDisableTiming));
    }
    const size_t esz = src.dt == PR_F64 ? 8 : 4;
    const int n_rows = p.nB, n_cols = p.nA;
    const size_t row_bytes = (size_t)n_cols * esz;
    int rows_per = (int)std::max<size_t>(1, kStageBytes / row_bytes);
    if ((n_rows + rows_per - 1) / rows_per > kStageMaxChunks) rows_per = (n_rows + kStageMaxChunks - 1) / kStageMaxChunks;
    const int sms = device_info().sms;
    PR_CUDA(cudaEventRecord(R.start, st));
    PR_CUDA(cudaStreamWaitEvent(R.copy, R.start, 0));
    const size_t pitch = (size_t)src.ldc * esz;
    for (int k = 0, r0 = 0; r0 < n_rows; ++k, r0 += rows_per) {
        const int rows = std::min(rows_per, n_rows - r0);
        PR_CUDA(cudaMemcpy2DAsync((char *)const_cast<void *>(src.C) + (size_t)r0 * pitch, pitch,
                                  (const char *)src.host + (size_t)r0 * pitch, pitch, row_bytes, rows,
                                  cudaMemcpyHostToDevice, R.copy));
        PR_CUDA(cudaEventRecord(R.done[k], R.copy));
        PR_CUDA(cudaStreamWaitEvent(st, R.done[k], 0));
        if (src.dt == PR_F64 && cb8) launch_quantise_rows<double, uint8_t>(src, p, r0, rows, eps, sms, st);
        else if (src.dt == PR_F64) launch_quantise_rows<double, uint16_t>(src, p, r0, rows, eps, sms, st);
        else if (cb8) launch_quantise_rows<float, uint8_t>(src, p, r0, rows, eps, sms, st);
        else launch_quantise_rows<float, uint16_t>(src, p, r0, rows, eps, sms, st);
        PR_CUDA(cudaGetLastError());
    }
    return PR_OK;
}

// Everything after the argument checks, shared by pr_assign, pr_assign_points
// and pr_assign_noalloc: p holds the workspace regions and sizes; this fills
// the scalars, then enqueues init, rounding, the phase loop, decode and finish.
pr_status launch_solve(Params &p, const CostSource &src, double eps, const PhaseCfg &cfg,
                       int32_t *row_to_col, int32_t *col_to_row, int32_t *y_col, double *cost,
                       pr_stats *stats, bool profile_ok, const char *who, cudaStream_t st) {
    const void *C = src.C;
    const pr_dtype dt = src.dt;
    const int64_t ldc = src.ldc;
    const int n_rows = p.nB, n_cols = p.nA;
    p.T = (int)floor(eps * (double)n_rows);
    const long long K = (long long)floor(1.0 / eps);
    p.phase_cap = ((long long)n_rows * (2 * K + 3)) / (p.T + 1) + 1;
    p.spin_limit = spin_limit_cycles();
    p.profile = 0;
    if (profile_ok) {
        const char *pf = getenv("PR_PROFILE");
        p.profile = (pf && *pf == '1') ? 1 : 0;
    }
    const bool cb8 = K <= kMaxCbar8;  // every cbar fits one byte
    const bool f7 = cb8 && K <= kMaxCbar7;  // and cbar + key < 256 on every real column

    const DeviceInfo &di = device_info();
    k_init<<<di.sms * 2, 256, 0, st>>>(p, row_to_col);
    PR_CUDA(cudaGetLastError());
    const long long groups = (long long)n_rows * (p.ldq >> 3);
    const long long want = groups / 256 + 1;
    const int qgrid = (int)(want < (long long)di.sms * 16 ? want : (long long)di.sms * 16);
    void *cbw = const_cast<void *>(p.cb);
    if (src.points) {
        const EpsSplit e = make_eps_split(eps);
        // 2-D and 3-D points with 16-byte-aligned columns take whole-vector loads
        const bool al = ((uintptr_t)src.XA % 16) == 0;
        const int D = al && (src.dim == 2 || src.dim == 3) ? src.dim : 0;
        if (D == 2) launch_points<2>(src, n_rows, n_cols, p, e, cb8, cbw, qgrid, st);
        else if (D == 3) launch_points<3>(src, n_rows, n_cols, p, e, cb8, cbw, qgrid, st);
        else launch_points<0>(src, n_rows, n_cols, p, e, cb8, cbw, qgrid, st);
    } else if (src.host) {
        const pr_status rc = stage_and_round(src, p, eps, cb8, st);
        if (rc != PR_OK) return rc;
    } else if (dt == PR_F64 && cb8)
        launch_quantise<double, uint8_t>((const double *)C, ldc, n_rows, n_cols, p.ldq, eps, (uint8_t *)cbw,
                                         &p.ctl->head, qgrid, st);
    else if (dt == PR_F64)
        launch_quantise<double, uint16_t>((const double *)C, ldc, n_rows, n_cols, p.ldq, eps, (uint16_t *)cbw,
                                          &p.ctl->head, qgrid, st);
    else if (cb8)
        launch_quantise<float, uint8_t>((const float *)C, ldc, n_rows, n_cols, p.ldq, eps, (uint8_t *)cbw,
                                        &p.ctl->head, qgrid, st);
    else
        launch_quantise<float, uint16_t>((const float *)C, ldc, n_rows, n_cols, p.ldq, eps, (uint16_t *)cbw,
                                         &p.ctl->head, qgrid, st);
    PR_CUDA(cudaGetLastError());

    const int chunk = cb8 ? kChunk<uint8_t> : kChunk<uint16_t>;
    const int chunks = (p.ldq + chunk - 1) / chunk;
    int warps_per_row = chunks < kWarps ? chunks : kWarps;
    int rows_per_group = kWarps / warps_per_row;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (profile_ok) kernel_events(&ev0, &ev1);
    if (ev0 && ev1) PR_CUDA(cudaEventRecord(ev0, st));
    const size_t row_bytes = (size_t)p.ldq * (cb8 ? 1 : 2);
    p.slot_bytes = (int)((row_bytes + 127) & ~size_t(127));
    const int kb = cb8 ? 1 : 2;  // bytes per key in the shared-memory copy
    const size_t slot_room = cfg.smem > slots_offset(p.ldq, kb) ? cfg.smem - slots_offset(p.ldq, kb) : 0;
    p.nslots = (int)std::min<size_t>((size_t)kWarps, slot_room / (size_t)p.slot_bytes);
    const bool cluster = p.rule <= PR_RULE_OFFSET && use_cluster(cfg, p.nslots, n_rows, K);
    if (p.rule == PR_RULE_SEQUENTIAL) {
        // the phase's keys live in shared memory, one per column (the size
        // was checked by pr_assign_rule)
        const size_t ksm = (size_t)p.ldq * (cb8 ? 1 : 2);
        const void *fn = cb8 ? (const void *)k_seq<uint8_t> : (const void *)k_seq<uint16_t>;
        PR_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ksm));
        Params pc = p;
        void *args[] = {(void *)&pc};
        PR_CUDA(cudaLaunchCooperativeKernel(fn, dim3(cfg.grid), dim3(kThreads), args, ksm, st));
    } else if (p.rule == PR_RULE_ISRAELI_ITAI) {
        if (!p.ii) return fail(PR_ERR_INVALID, "%s: the Israeli-Itai rule needs a workspace", who);
        // the rule's state: 8-byte words first, then the int arrays
        IIWork w;
        unsigned long long *q = (unsigned long long *)p.ii;
        w.cp = q;
        w.cin = q + n_cols;
        w.rin = q + 2 * (size_t)n_cols;
        int *r = (int *)(q + 2 * (size_t)n_cols + n_rows);
        w.mB = r;
        w.act = r + n_rows;
        w.mate = r + 2 * (size_t)n_rows;
        w.rp = r + 3 * (size_t)n_rows;
        w.rc = r + 4 * (size_t)n_rows;
        w.mA = r + 5 * (size_t)n_rows;
        w.taken = w.mA + n_cols;
        w.cc = w.taken + n_cols;
        Params pc = p;
        void *args[] = {(void *)&pc, (void *)&w};
        const void *fn = cb8 ? (const void *)k_ii<uint8_t> : (const void *)k_ii<uint16_t>;
        PR_CUDA(cudaLaunchCooperativeKernel(fn, dim3(cfg.grid), dim3(kThreads), args, 0, st));
    } else if (cluster) {
        cudaLaunchConfig_t c = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cfg.cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        c.gridDim = dim3(cfg.cluster);
        c.blockDim = dim3(kThreads);
        c.dynamicSmemBytes = slots_offset(p.ldq, kb) + (size_t)p.nslots * p.slot_bytes;
        c.stream = st;
        c.attrs = at;
        c.numAttrs = 1;
        Params pc = p;
        void *args[] = {(void *)&pc, (void *)&warps_per_row, (void *)&rows_per_group};
        PR_CUDA(cudaLaunchKernelExC(&c, phase_kernel(cb8, true, true, f7, p.rule != 0), args));
    } else {
        Params pc = p;
        void *args[] = {(void *)&pc, (void *)&warps_per_row, (void *)&rows_per_group};
        const bool sl = use_slots_in_grid(p.nslots);
        const void *fn = phase_kernel(cb8, false, sl, f7, p.rule != 0);
        const size_t smem = sl ? slots_offset(p.ldq, kb) + (size_t)p.nslots * p.slot_bytes : smem_bytes(p.ldq, kb);
        PR_CUDA(cudaLaunchCooperativeKernel(fn, dim3(cfg.grid), dim3(kThreads), args, smem, st));
    }
    if (ev0 && ev1) PR_CUDA(cudaEventRecord(ev1, st));

    k_decode<<<di.sms * 2, 256, 0, st>>>(p, row_to_col, col_to_row, y_col);
    PR_CUDA(cudaGetLastError());
    // completion scratch: the first CTA's list region (free after the loop)
    int *free_b = p.lists;
    int *free_a = p.lists + n_rows;
    if (src.points)
        k_finish<PointsCost><<<1, kFinThreads, 0, st>>>(p, PointsCost{src.XA, src.XB, src.dim, src.squared},
                                                         row_to_col, col_to_row, free_b, free_a, cost);
    else if (dt == PR_F64)
        k_finish<MatrixCost<double>><<<1, kFinThreads, 0, st>>>(p, MatrixCost<double>{(const double *)C, ldc},
                                                                row_to_col, col_to_row, free_b, free_a, cost);
    else
        k_finish<MatrixCost<float>><<<1, kFinThreads, 0, st>>>(p, MatrixCost<float>{(const float *)C, ldc},
                                                               row_to_col, col_to_row, free_b, free_a, cost);
    PR_CUDA(cudaGetLastError());

    if (stats) {
        Ctl h;
        PR_CUDA(cudaMemcpyAsync(&h, p.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        PR_CUDA(cudaStreamSynchronize(st));
        stats->phases = h.phases;
        stats->rounds = h.rounds;
        stats->bytes_scanned = (int64_t)h.bytes;
        stats->rows_scanned = (int64_t)h.rows;
        stats->cells_examined = (int64_t)h.cells;
        stats->free_at_stop = h.free_at_stop;
        stats->threshold = p.T;
        stats->loop_ctas = cluster ? cfg.cluster : cfg.grid;
        stats->loop_cluster = cluster ? 1 : 0;
        stats->barriers = (int64_t)h.barriers;
        if (h.head.err != 0)
            return fail((pr_status)h.head.err, "%s: device reported %s", who,
                        pr_status_string((pr_status)h.head.err));
    }
    return PR_OK;
}

}  // namespace
}  // namespace prot

using namespace prot;

extern "C" size_t pr_assign_workspace(int32_t n_rows, int32_t n_cols) {
    if (n_rows < 1 || n_cols < n_rows || n_cols > (1 << 24) - 1) return 0;
    PhaseCfg cfg;
    if (phase_cfg(cfg) != PR_OK) cfg.grid = kMaxGrid;  // no device: the largest grid
    return make_layout(n_rows, n_cols, cfg.grid).total;
}

namespace prot {
namespace {

// The address the kernels read a cost matrix through: device or managed
// memory as it is; pinned (page-locked) host memory through its mapping
// into the device address space, so the rounding kernel reads it in place
// over the host link.  Any other host memory is refused here, before
// anything is enqueued (a kernel would fault on it).
pr_status device_view(const void *C, const void **out, const char *who) {
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, C);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PR_ERR_INVALID, "%s: C is not memory the CUDA runtime knows", who);
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        *out = C;
        return PR_OK;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *out = a.devicePointer;
        return PR_OK;
    }
    return fail(PR_ERR_INVALID, "%s: C must be device memory or pinned host memory", who);
}

// pr_assign and pr_assign_points after their own source checks: sizes, eps,
// workspace, then the solve.
pr_status assign_common(const CostSource &src, int32_t n_rows, int32_t n_cols, double eps,
                        int32_t *row_to_col, int32_t *col_to_row, int32_t *y_row, int32_t *y_col,
                        double *cost, pr_stats *stats, void *ws, size_t ws_bytes, void *stream,
                        const char *who, int rule = PR_RULE_LOWEST) {
    if (!row_to_col || !col_to_row || !y_row || !y_col || !cost)
        return fail(PR_ERR_INVALID, "%s: NULL pointer argument", who);
    if (n_rows < 1 || n_cols < n_rows || n_cols > (1 << 24) - 1)
        return fail(PR_ERR_INVALID, "%s: need 1 <= n_rows <= n_cols < 2^24", who);
    if (!(eps > 0.0 && eps < 1.0) || floor(1.0 / eps) > 32766.0)
        return fail(PR_ERR_INVALID, "%s: need 0 < eps < 1 and floor(1/eps) <= 32766", who);
    PhaseCfg cfg;
    pr_status rc = phase_cfg(cfg);
    if (rc != PR_OK) return rc;
    const Layout L = make_layout(n_rows, n_cols, cfg.grid);
    if (smem_bytes(L.ldq) > cfg.smem)
        // each column costs 2 bytes of key copy and 1/8 byte of taken set
        return fail(PR_ERR_INVALID, "%s: n_cols = %d exceeds the shared-memory key copy (max %d)", who,
                    n_cols, (int)((cfg.smem - smem_bytes(0)) * 8 / 17) & ~31);
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < L.total)
        return fail(PR_ERR_WORKSPACE, "%s: workspace NULL, not 256-byte aligned or < %zu bytes", who,
                    L.total);
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;

    Params p;
    p.ctl = (Ctl *)(w + L.ctl);
    p.cb = w + L.cb;
    p.ka = (uint16_t *)(w + L.ka);
    p.y_b = y_row;
    p.prop = (unsigned long long *)(w + L.prop);
    p.won = (unsigned *)(w + L.won);
    p.won_words = L.won_words;
    p.pool = (int2 *)(w + L.pool);
    p.lists = (int *)(w + L.lists);
    p.list_stride = L.list_stride;
    p.nB = n_rows;
    p.nA = n_cols;
    p.ldq = L.ldq;
    p.rule = rule;
    p.ii = w + L.ii;
    return launch_solve(p, src, eps, cfg, row_to_col, col_to_row, y_col, cost, stats, true, who, st);
}

}  // namespace
}  // namespace prot

extern "C" pr_status pr_assign(const void *C, pr_dtype dt, int64_t ldc, int32_t n_rows,
                               int32_t n_cols, double eps, int32_t *row_to_col,
                               int32_t *col_to_row, int32_t *y_row, int32_t *y_col, double *cost,
                               pr_stats *stats, void *ws, size_t ws_bytes, void *stream) {
    if (!C) return fail(PR_ERR_INVALID, "pr_assign: NULL pointer argument");
    if (dt != PR_F32 && dt != PR_F64) return fail(PR_ERR_INVALID, "pr_assign: bad dtype");
    if (ldc < n_cols) return fail(PR_ERR_INVALID, "pr_assign: ldc < n_cols");
    CostSource src;
    if (row_to_col && col_to_row && y_row && y_col && cost) {  // NULL outputs: reported below
        const pr_status rc = device_view(C, &src.C, "pr_assign");
        if (rc != PR_OK) return rc;
    }
    src.dt = dt;
    src.ldc = ldc;
    return assign_common(src, n_rows, n_cols, eps, row_to_col, col_to_row, y_row, y_col, cost, stats, ws,
                         ws_bytes, stream, "pr_assign");
}

extern "C" pr_status pr_assign_within(const void *C, pr_dtype dt, int64_t ldc, int32_t n_rows, int32_t n_cols,
                                      double delta, int32_t *row_to_col, int32_t *col_to_row, int32_t *y_row,
                                      int32_t *y_col, double *cost, pr_stats *stats, void *ws, size_t ws_bytes,
                                      void *stream) {
    // Sec. 1: the 3 eps n routine run with eps = delta / 3 is a delta n approximation
    if (!(delta > 0.0 && delta < 3.0)) return fail(PR_ERR_INVALID, "pr_assign_within: need 0 < delta < 3");
    return pr_assign(C, dt, ldc, n_rows, n_cols, delta / 3.0, row_to_col, col_to_row, y_row, y_col, cost, stats,
                     ws, ws_bytes, stream);
}

extern "C" pr_status pr_assign_rule(pr_rule rule, const void *C, pr_dtype dt, int64_t ldc, int32_t n_rows,
                                    int32_t n_cols, double eps, int32_t *row_to_col, int32_t *col_to_row,
                                    int32_t *y_row, int32_t *y_col, double *cost, pr_stats *stats, void *ws,
                                    size_t ws_bytes, void *stream) {
    if (rule != PR_RULE_LOWEST && rule != PR_RULE_OFFSET && rule != PR_RULE_ISRAELI_ITAI &&
        rule != PR_RULE_SEQUENTIAL)
        return fail(PR_ERR_INVALID, "pr_assign_rule: bad rule");
    if (!C) return fail(PR_ERR_INVALID, "pr_assign_rule: NULL pointer argument");
    if (dt != PR_F32 && dt != PR_F64) return fail(PR_ERR_INVALID, "pr_assign_rule: bad dtype");
    if (rule == PR_RULE_SEQUENTIAL && eps > 0.0 && eps < 1.0) {
        // the phase's keys live in shared memory, one byte (floor(1/eps) <=
        // 252) or two per column
        const size_t kb = (long long)floor(1.0 / eps) <= kMaxCbar8 ? 1 : 2;
        if ((((size_t)n_cols + 15) & ~(size_t)15) * kb > kSeqMaxKeyBytes)
            return fail(PR_ERR_INVALID, "pr_assign_rule: the sequential rule takes at most %zu columns at this eps",
                        kSeqMaxKeyBytes / kb);
    }
    if (ldc < n_cols) return fail(PR_ERR_INVALID, "pr_assign_rule: ldc < n_cols");
    CostSource src;
    if (row_to_col && col_to_row && y_row && y_col && cost) {  // NULL outputs: reported below
        const pr_status rc = device_view(C, &src.C, "pr_assign_rule");
        if (rc != PR_OK) return rc;
    }
    src.dt = dt;
    src.ldc = ldc;
    return assign_common(src, n_rows, n_cols, eps, row_to_col, col_to_row, y_row, y_col, cost, stats, ws,
                         ws_bytes, stream, "pr_assign_rule", (int)rule);
}

extern "C" pr_status pr_assign_staged(const void *C_host, void *C_dev, pr_dtype dt, int64_t ldc, int32_t n_rows,
                                      int32_t n_cols, double eps, int32_t *row_to_col, int32_t *col_to_row,
                                      int32_t *y_row, int32_t *y_col, double *cost, pr_stats *stats, void *ws,
                                      size_t ws_bytes, void *stream) {
    if (!C_host || !C_dev) return fail(PR_ERR_INVALID, "pr_assign_staged: NULL pointer argument");
    if (dt != PR_F32 && dt != PR_F64) return fail(PR_ERR_INVALID, "pr_assign_staged: bad dtype");
    if (ldc < n_cols) return fail(PR_ERR_INVALID, "pr_assign_staged: ldc < n_cols");
    cudaPointerAttributes ah, ad;
    if (cudaPointerGetAttributes(&ah, C_host) != cudaSuccess ||
        cudaPointerGetAttributes(&ad, C_dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(PR_ERR_INVALID, "pr_assign_staged: a pointer the CUDA runtime does not know");
    }
    if (ah.type != cudaMemoryTypeHost && ah.type != cudaMemoryTypeUnregistered)
        return fail(PR_ERR_INVALID, "pr_assign_staged: C_host must be host memory");
    if (ad.type != cudaMemoryTypeDevice)
        return fail(PR_ERR_INVALID, "pr_assign_staged: C_dev must be device memory");
    CostSource src;
    src.C = C_dev;
    src.host = C_host;
    src.dt = dt;
    src.ldc = ldc;
    return assign_common(src, n_rows, n_cols, eps, row_to_col, col_to_row, y_row, y_col, cost, stats, ws,
                         ws_bytes, stream, "pr_assign_staged");
}

extern "C" pr_status pr_assign_points(const float *XA, const float *XB, int32_t dim, pr_metric metric,
                                      int32_t n_rows, int32_t n_cols, double eps, int32_t *row_to_col,
                                      int32_t *col_to_row, int32_t *y_row, int32_t *y_col, double *cost,
                                      pr_stats *stats, void *ws, size_t ws_bytes, void *stream) {
    if (!XA || !XB) return fail(PR_ERR_INVALID, "pr_assign_points: NULL point pointer");
    if (dim < 1 || dim > 4096) return fail(PR_ERR_INVALID, "pr_assign_points: need 1 <= dim <= 4096");
    if (metric != PR_SQEUCLIDEAN && metric != PR_EUCLIDEAN)
        return fail(PR_ERR_INVALID, "pr_assign_points: bad metric");
    CostSource src;
    src.XA = XA;
    src.XB = XB;
    src.dim = dim;
    src.squared = metric == PR_SQEUCLIDEAN ? 1 : 0;
    src.points = true;
    return assign_common(src, n_rows, n_cols, eps, row_to_col, col_to_row, y_row, y_col, cost, stats, ws,
                         ws_bytes, stream, "pr_assign_points");
}

// ---------------------------------------------------------------------------
// pr_assign_noalloc: the pr_assign solve for callers that cannot allocate
// device memory.  Its scratch is one file-scope device array of fixed size.
// ---------------------------------------------------------------------------
namespace prot {
namespace {

constexpr int kNoAllocMaxN = 1024;  // largest n_cols (and so n_rows) accepted

// Bytes the scratch layout below needs for n_rows = n_cols = kNoAllocMaxN,
// rounded up; checked against the real layout on every call.
constexpr size_t kNoAllocBytes = (size_t)2304 * 1024;

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocLayout {
    size_t ctl, cb, ka, prop, won, pool, lists, total;
    int ldq, won_words;
};

// The regions k_init .. k_finish use.  The per-CTA proposal-list overflow is
// absent: with n_rows <= 1024 every list fits the shared-memory part.
NoAllocLayout make_noalloc_layout(int nB, int nA) {
    NoAllocLayout L;
    Carver c;
    L.ldq = (nA + 15) & ~15;  // rows start on 16 bytes in either storage type
    L.ctl = c.take<Ctl>(1);
    L.cb = c.take<uint16_t>((size_t)nB * L.ldq);  // room for the uint16 form
    L.ka = c.take<uint16_t>(L.ldq);
    L.prop = c.take<unsigned long long>((size_t)nA);
    L.won_words = (nA + 31) / 32;
    L.won = c.take<unsigned>(3 * (size_t)L.won_words);
    L.pool = c.take<int2>(2 * (size_t)nB);
    L.lists = c.take<int>(2 * (size_t)nB);  // completion scratch
    L.total = c.total();
    return L;
}

// Device address of the scratch array for the current device.  It is looked
// up on every call (cudaGetSymbolAddress must run with that device current;
// it allocates nothing), so no address outlives a reload of the module.
pr_status noalloc_scratch(char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = (char *)p;
    return PR_OK;
}

}  // namespace
}  // namespace prot

extern "C" pr_status pr_assign_noalloc(const void *C, pr_dtype dt, int64_t ldc, int32_t n_rows,
                                       int32_t n_cols, double eps, int32_t *row_to_col,
                                       int32_t *col_to_row, int32_t *y_row, int32_t *y_col,
                                       double *cost, pr_stats *stats, void *stream) {
    if (!C || !row_to_col || !col_to_row || !y_row || !y_col || !cost)
        return fail(PR_ERR_INVALID, "pr_assign_noalloc: NULL pointer argument");
    if (dt != PR_F32 && dt != PR_F64) return fail(PR_ERR_INVALID, "pr_assign_noalloc: bad dtype");
    if (n_rows < 1 || n_cols < n_rows)
        return fail(PR_ERR_INVALID, "pr_assign_noalloc: need 1 <= n_rows <= n_cols");
    if (n_cols > kNoAllocMaxN)
        return fail(PR_ERR_INVALID,
                    "pr_assign_noalloc: n_cols = %d exceeds the built-in scratch limit of %d "
                    "(use pr_assign with a caller workspace)",
                    n_cols, kNoAllocMaxN);
    if (ldc < n_cols) return fail(PR_ERR_INVALID, "pr_assign_noalloc: ldc < n_cols");
    if (!(eps > 0.0 && eps < 1.0) || floor(1.0 / eps) > 32766.0)
        return fail(PR_ERR_INVALID, "pr_assign_noalloc: need 0 < eps < 1 and floor(1/eps) <= 32766");
    // the same source check as pr_assign: pageable host memory is refused
    // here, pinned host memory is read through its device mapping
    const void *Cd = nullptr;
    pr_status vrc = device_view(C, &Cd, "pr_assign_noalloc");
    if (vrc != PR_OK) return vrc;
    const NoAllocLayout L = make_noalloc_layout(n_rows, n_cols);
    if (L.total > kNoAllocBytes) return fail(PR_ERR_WORKSPACE, "pr_assign_noalloc: scratch layout too large");
    PhaseCfg cfg;
    pr_status rc = phase_cfg(cfg);
    if (rc != PR_OK) return rc;
    char *w = nullptr;
    rc = noalloc_scratch(&w);
    if (rc != PR_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    Params p;
    p.ctl = (Ctl *)(w + L.ctl);
    p.cb = w + L.cb;
    p.ka = (uint16_t *)(w + L.ka);
    p.y_b = y_row;
    p.prop = (unsigned long long *)(w + L.prop);
    p.won = (unsigned *)(w + L.won);
    p.won_words = L.won_words;
    p.pool = (int2 *)(w + L.pool);
    p.lists = (int *)(w + L.lists);
    p.list_stride = 0;  // no overflow region: never addressed for n_rows <= 1024
    p.nB = n_rows;
    p.nA = n_cols;
    p.ldq = L.ldq;
    CostSource src;
    src.C = Cd;
    src.dt = dt;
    src.ldc = ldc;
    return launch_solve(p, src, eps, cfg, row_to_col, col_to_row, y_col, cost, stats, false,
                        "pr_assign_noalloc", st);
}
