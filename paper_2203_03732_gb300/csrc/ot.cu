// ot.cu -- pr_ot: the optimal-transport form of Sec. 4 on one GB300.
//
// Sec. 4 scales the masses by theta = 4n/eps, rounds supplies down and
// demands up, and runs the matching algorithm of Sec. 2.2 on the unit copies,
// keeping every free supply copy's dual raised to the largest dual among its
// siblings.  The copies are handled as clusters:
//   supply b: F_b (dual of its free copies, the largest of its copies),
//             f_b (free copies);
//   demand a: keys k = -y in {kmin_a, kmin_a + 1} (Lemma 4.1): clo_a copies
//             at kmin_a, chi_a at kmin_a + 1.
// eps-feasibility of a free copy against a's kmin copies makes a's kmin
// cluster the only one that can be admissible, and (a, b) is admissible iff
// cbar(b,a) + kmin_a == F_b - 1 -- the assignment test with k(a) = kmin_a.
//
// Matched copy counts live in one list per demand a: entries (b, lo, hi),
// ascending b, each b at most once, where lo counts b's copies matched to a's
// copies at key kmin_a (a's "lo" cluster) and hi those at kmin_a + 1.  A
// grant adds to b's hi count (a new entry is inserted in order); an eviction
// takes lo counts from the end of the list (highest supply index first).
// When the lo cluster runs out (every match in it was evicted, or it held
// a's free copies) the clusters shift: every entry's hi count becomes its lo
// count, and entries left with none are dropped.  A list starts in a fixed
// slot of 32 entries; a longer list moves to a slot of twice the size from a
// shared arena (bump allocation, never freed; a list keeps its slot).  The
// lists hold about as many entries as there are matched (supply, demand)
// pairs (measured: 0.9 to 1.5 x (n_sup + n_dem) at their largest), so the
// storage is O(n_sup + n_dem), not n_sup x n_dem.  The plan's matched
// entries are read straight from the lists after the loop.
//
// One phase (B' = supply vertices with free copies), steps of k_ot_loop (one
// cooperative launch; a grid barrier with a summed payload after each step):
//   ot_phase_start  r_b = f_b, flags, the free-copy total for the stop test
//   round R: ot_propose  every searching b proposes (atomicMax on the column
//                        word) to the lowest admissible a >= its resume
//                        column with unmatched lo copies left;
//            ot_grant    a's lowest proposer b gets g = min(r_b, avail_a)
//                        copies; partners of matched lo copies are evicted,
//                        highest supply index first (step II)
//   ot_phase_end    F_b += 1 for b in B' left with unplaced copies (III b);
//                   clusters shift up where the lo cluster is empty (III a)
// Nothing in a solve waits for the host: errors found on the device (masses,
// costs, the loop, the plan capacity) are recorded in the workspace head, the
// kernels after them return at once, and the host reads the head only when
// the caller asks for stats (or later through pr_ws_status).
//
// Plan and fix-up (a reading: the paper defers this part to another paper):
// mass(b,a) = matched copies / theta; a demand that received more than mu_a
// gives the excess back from its highest supply index; each supply's unsent
// remainder is routed north-west-corner style (b ascending, a ascending) into
// the remaining demand capacity.  The FP64 arithmetic of the fix-up follows
// one fixed order (ascending b per demand, ascending a per supply), so the
// residuals are reproducible bit for bit.  The north-west rule then runs on
// the residuals rounded down to whole units of 2^-62, in exact integers: an
// allocation starts wherever a supply's or a demand's run of units starts in
// the two prefix sums, so every allocation is found in parallel (a merge of
// the two sorted lists of run starts) with the serial walk's result.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "prot_internal.cuh"
#include "quantise.cuh"
#include "scan_common.cuh"

namespace prot {
namespace {

constexpr int kOtThreads = 256;
constexpr int kOtUnroll = 4;  // 2 KiB warp chunks (swept 3, 4, 8 at 10k x 10k)
constexpr int kFlagSearching = 1, kFlagInBp = 2;
constexpr int kCostCtas = 64;  // CTAs of the cost sum (a constant: same order on every device)
constexpr int kListSlot = 32;  // entries of a demand's first list slot (one per lane of a warp)

struct OCtl {
    WsHead head;
    unsigned long long bar[4];  // payload barrier slots of k_ot_loop
    long long phases, rounds, free_at_stop, threshold;
    int nnz;                    // plan entries from the matched copies
    int n_nw;                   // north-west corner allocations
    int n_extra;                // allocations on pairs without matched copies
    int pad;
    long long bytes;
    unsigned long long mass_units[2];  // sum of floor(m 2^32) over supplies, demands
    unsigned cost_done;                // CTAs of k_fix_cost that have finished
    unsigned arena_top;                // list entries taken from the arena so far
    double cost_part[kCostCtas];       // their partial sums
};

struct OLayout {
    size_t ctl, cb, key, S, D, F, f, r, ptr, flag, kmin, clo, chi, avail, granted, prop;
    size_t eb, elo, ehi, seg_off, seg_cap, seg_len;
    size_t nnz_a, off_a, trim_b, trim_t, q, rres, cnt_b, off_b, bsort_a, nw_flag,
        nw_off, nw_b, nw_a, nw_t, nw_pr, nw_pq, nw_pos, total;
    int ldq;
    long long arena;      // entries of the list arena
    long long list_cap;   // entries of all list storage: n_dem first slots + the arena
};

// The arena holds the lists that outgrow their first slot.  A list of L
// entries has taken at most 4L arena entries (slots of 64, 128, ... up to 2L),
// and the lists together hold about (n_sup + n_dem) entries or fewer, so 8 x
// (n_sup + n_dem) leaves room; a solve that needs more reports
// PR_ERR_CAPACITY.
inline long long ot_arena_entries(int nB, int nA) { return 8ll * ((long long)nB + nA) + 4096; }

OLayout make_olayout(int nB, int nA) {
    OLayout L;
    Carver c;
    L.ldq = (nA + 15) & ~15;  // rows start on 16 bytes in either storage type
    L.ctl = c.take<OCtl>(1);
    L.cb = c.take<uint16_t>((size_t)nB * L.ldq);
    L.key = c.take<uint16_t>(L.ldq);
    L.S = c.take<int>(nB);
    L.D = c.take<int>(nA);
    L.F = c.take<int>(nB);
    L.f = c.take<int>(nB);
    L.r = c.take<int>(nB);
    L.ptr = c.take<int>(nB);
    L.flag = c.take<int>(nB);
    L.kmin = c.take<int>(nA);
    L.clo = c.take<int>(nA);
    L.chi = c.take<int>(nA);
    L.avail = c.take<int>(nA);
    L.granted = c.take<int>(nA);
    L.prop = c.take<unsigned long long>(nA);
    L.arena = ot_arena_entries(nB, nA);
    L.list_cap = (long long)nA * kListSlot + L.arena;
    L.eb = c.take<int>((size_t)L.list_cap);
    L.elo = c.take<int>((size_t)L.list_cap);
    L.ehi = c.take<int>((size_t)L.list_cap);
    L.seg_off = c.take<int>(nA);
    L.seg_cap = c.take<int>(nA);
    L.seg_len = c.take<int>(nA);
    L.nnz_a = c.take<int>(nA);
    L.off_a = c.take<int>((size_t)nA + 1);
    L.trim_b = c.take<int>(nA);
    L.trim_t = c.take<double>(nA);
    L.q = c.take<double>(nA);
    L.rres = c.take<double>(nB);
    L.cnt_b = c.take<int>(nB);
    L.off_b = c.take<int>((size_t)nB + 1);
    L.bsort_a = c.take<int>((size_t)L.list_cap);  // the plan's matched entries, by supply
    L.nw_flag = c.take<int>((size_t)nB + nA);
    L.nw_off = c.take<int>((size_t)nB + nA + 1);
    L.nw_b = c.take<int>((size_t)nB + nA);
    L.nw_a = c.take<int>((size_t)nB + nA);
    L.nw_t = c.take<double>((size_t)nB + nA);
    L.nw_pr = c.take<unsigned long long>(nB);
    L.nw_pq = c.take<unsigned long long>(nA);
    L.nw_pos = c.take<int>((size_t)nB + nA);
    L.total = c.total();
    return L;
}

struct OParams {
    OCtl *ctl;
    const void *cb;  // uint8_t or uint16_t [nB][ldq] (bytes when floor(1/eps) <= 252)
    void *key;       // k = kmin_a per column, in the same type (padding 0xFF / 0x8000)
    int *S, *D, *F, *f, *r, *ptr, *flag;
    int *kmin, *clo, *chi, *avail, *granted;
    unsigned long long *prop;
    // per-demand lists: entry i of a's list is (eb, elo, ehi)[seg_off[a] + i],
    // i < seg_len[a] <= seg_cap[a]; arena slots start at n_dem * kListSlot
    int *eb, *elo, *ehi;
    int *seg_off, *seg_cap, *seg_len;
    long long list_cap;
    int nB, nA, ldq;
};

// S_b = floor(theta nu_b), D_a = ceil(theta mu_a) (Sec. 4), one FP64 product
// each.  Also sums floor(m 2^32) per side, exactly (each term < 2^33): the
// host refuses a side whose sum reaches 1.5 * 2^32, and a mass of 2 or more
// is refused here, so the fix-up's 2^-62 units and their totals stay below
// 2^63.
__global__ void k_ot_counts(const double *nu, const double *mu, int nB, int nA, double theta,
                            int *S, int *D, OCtl *ctl) {
    const int stride = gridDim.x * blockDim.x;
    unsigned long long us = 0, ud = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nB + nA; i += stride) {
        const bool sup = i < nB;
        const double m = sup ? nu[i] : mu[i - nB];
        const double v = sup ? floor(__dmul_rn(theta, m)) : ceil(__dmul_rn(theta, m));
        if (!(m >= 0.0) || !(m < 2.0) || !(v <= 2147483647.0)) {
            record_error(&ctl->head, PR_ERR_INVALID);
            continue;
        }
        const unsigned long long u = __double2ull_rz(__dmul_rn(m, 0x1p32));
        if (sup) {
            S[i] = (int)v;
            us += u;
        } else {
            D[i - nB] = (int)v;
            ud += u;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        us += __shfl_down_sync(0xFFFFFFFFu, us, o);
        ud += __shfl_down_sync(0xFFFFFFFFu, ud, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (us) atomicAdd(&ctl->mass_units[0], us);
        if (ud) atomicAdd(&ctl->mass_units[1], ud);
    }
}

// Runs after k_ot_counts (stream order), so the mass sums are complete: a
// side whose floor(m 2^32) sum to 1.5 * 2^32 or more is refused here.
template <class CB>
__global__ void k_ot_init(OParams p) {
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0 && (p.ctl->mass_units[0] >= (3ull << 31) || p.ctl->mass_units[1] >= (3ull << 31)))
        record_error(&p.ctl->head, PR_ERR_INVALID);
    for (int b = t0; b < p.nB; b += stride) {
        p.F[b] = 1;
        p.f[b] = p.S[b];
        p.r[b] = 0;
        p.ptr[b] = 0;
        p.flag[b] = 0;
    }
    for (int a = t0; a < p.ldq; a += stride) {
        static_cast<CB *>(p.key)[a] = a < p.nA ? (CB)0 : (CB)(sizeof(CB) == 1 ? 0xFF : kPadKey);
        if (a >= p.nA) continue;
        p.kmin[a] = 0;
        p.clo[a] = p.D[a];
        p.chi[a] = 0;
        p.avail[a] = p.D[a];
        p.granted[a] = 0;
        p.prop[a] = word_of(0, -1);
        p.seg_off[a] = a * kListSlot;  // every list starts empty in its first slot
        p.seg_cap[a] = kListSlot;
        p.seg_len[a] = 0;
    }
}

__global__ void k_ot_ctl_init(OCtl *c) {
    memset(c, 0, sizeof(OCtl));
    c->head.magic = kWsMagic;
}

// Sum over the CTA of one value per thread (every thread gets the sum).
__device__ __forceinline__ unsigned long long cta_sum(unsigned long long v) {
    __shared__ unsigned long long acc;
    __syncthreads();
    if (threadIdx.x == 0) acc = 0;
    __syncthreads();
    if (v) atomicAdd(&acc, v);
    __syncthreads();
    return acc;
}

// Phase start: r_b = f_b, B' = {b : f_b > 0}; returns this thread's free copies.
__device__ __forceinline__ unsigned long long ot_phase_start(const OParams &p) {
    unsigned long long mine = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < p.nB; b += gridDim.x * blockDim.x) {
        const int fb = ld_relaxed_s32(p.f + b);  // evictions add to it from any CTA
        p.r[b] = fb;
        p.flag[b] = fb > 0 ? (kFlagSearching | kFlagInBp) : 0;
        p.ptr[b] = 0;
        mine += (unsigned long long)fb;
    }
    return mine;
}

// Warp per searching supply vertex: the lowest a >= ptr with
// cbar + kmin_a == F_b - 1 and avail_a > 0.
// Returns this thread's proposals (lane 0 of each warp counts its rows).
// F7: floor(1/eps) <= 125, so every sum of a real column's cbar and key
// stays below 256 and the byte pre-test is one plain add (may_match<true>).
template <class CB, bool F7>
__device__ __forceinline__ unsigned ot_propose(const OParams &p, unsigned R, unsigned long long &bytes_out) {
    constexpr int W = 16 / (int)sizeof(CB);  // columns per 16-byte load
    constexpr unsigned kAll = W == 16 ? 0xFFFFu : 0xFFu;
    constexpr int kChunkW = 32 * W * kOtUnroll;
    unsigned props = 0;
    const int lane = threadIdx.x & 31;
    const int warp_g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const CB *key = static_cast<const CB *>(p.key);
    unsigned long long bytes = 0;
    // a row's flag, dual and resume column are loaded together, and the next
    // row's while this one is scanned (only this warp writes them in this
    // step; other CTAs wrote them in earlier steps, so the loads go to L2)
    int nfl = 0, nF = 0, nst = 0;
    if (warp_g < p.nB) {
        nfl = ld_relaxed_s32(p.flag + warp_g);
        nF = ld_relaxed_s32(p.F + warp_g);
        nst = ld_relaxed_s32(p.ptr + warp_g);
    }
    for (int b = warp_g; b < p.nB; b += nwarps) {
        const int fl = nfl, Fb = nF, start = nst;
        if (b + nwarps < p.nB) {
            nfl = ld_relaxed_s32(p.flag + b + nwarps);
            nF = ld_relaxed_s32(p.F + b + nwarps);
            nst = ld_relaxed_s32(p.ptr + b + nwarps);
        }
        if (!(fl & kFlagSearching)) continue;
        const uint32_t tgt = (uint32_t)(Fb - 1);
        const uint32_t t2 = W == 8 ? (tgt | (tgt << 16)) : tgt * 0x01010101u;
        const CB *row = static_cast<const CB *>(p.cb) + (size_t)b * p.ldq;
        int found = -1;
        for (int c0 = start & ~(W - 1); c0 < p.ldq && found < 0; c0 += kChunkW) {
            uint4 cv[kOtUnroll];
#pragma unroll
            for (int u = 0; u < kOtUnroll; ++u) {
                const int idx = c0 + u * 32 * W + lane * W;
                cv[u] = idx < p.ldq ? ld_nc_na_v4(row + idx) : make_uint4(0, 0, 0, 0);
            }
            bytes += sizeof(CB) * (unsigned long long)min(kChunkW, p.ldq - c0);
            for (int u = 0; u < kOtUnroll && found < 0; ++u) {
                const int idx = c0 + u * 32 * W + lane * W;
                unsigned m = 0;
                if (idx < p.ldq) {
                    const uint4 kv = *reinterpret_cast<const uint4 *>(key + idx);
                    m = W == 8 ? eq_mask(make_uint4(cv[u].x + kv.x, cv[u].y + kv.y, cv[u].z + kv.z, cv[u].w + kv.w), t2)
                               : eq_mask8<F7>(cv[u], kv, t2);
                }
                const int lo = start - idx;
                if (lo > 0) m &= lo >= W ? 0u : (kAll << lo) & kAll;
                // every lane checks its lowest candidate's copies at once;
                // the lowest lane with copies wins once no lower lane holds
                // a candidate (lanes are in column order)
                for (;;) {
                    if (__ballot_sync(0xFFFFFFFFu, m != 0) == 0) break;
                    const int a_mine = idx + __ffs(m) - 1;
                    const bool ok = m != 0 && ld_relaxed_s32(p.avail + a_mine) > 0;
                    const unsigned okm = __ballot_sync(0xFFFFFFFFu, ok);
                    if (!ok && m) m &= m - 1;
                    if (okm) {
                        const int L = __ffs(okm) - 1;
                        if ((__ballot_sync(0xFFFFFFFFu, m != 0) & ((1u << L) - 1)) == 0) {
                            found = __shfl_sync(0xFFFFFFFFu, a_mine, L);
                            break;
                        }
                    }
                }
            }
        }
        if (lane == 0) {
            if (found >= 0) {
                atomicMax(p.prop + found, word_of(R, b));
                p.ptr[b] = found;
                ++props;
            } else {
                atomicAnd(p.flag + b, ~kFlagSearching);
            }
        }
    }
    if (lane == 0) bytes_out += bytes;
    return props;
}

// ---------------------------------------------------------------------------
// Per-demand lists (warp operations; only the grant or the phase end of
// demand a touches a's list, one warp at a time)
// ---------------------------------------------------------------------------
// Step (II): take `need` lo copies from a's list, highest supply index first
// (the end of the list); each copy taken rejoins its supply's free copies.
__device__ __forceinline__ void list_evict(const OParams &p, int a, int need, int lane) {
    const int off = p.seg_off[a], n = p.seg_len[a];
    int taken = 0;  // lo copies of the entries above this chunk
    for (int top = n - 1; top >= 0 && taken < need; top -= 32) {
        const int i = top - lane;  // lane 0: the highest remaining entry
        const int c = i >= 0 ? p.elo[off + i] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        int t = need - (taken + incl - c);
        t = t < 0 ? 0 : (t > c ? c : t);
        if (t > 0) {
            p.elo[off + i] = c - t;
            atomicAdd(p.f + p.eb[off + i], t);
        }
        taken += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
}

// g copies of b matched to a's hi cluster: added to b's entry, or a new entry
// inserted in ascending order (the list moves to a slot twice its size from
// the arena when full).  Returns false when the arena is spent.
__device__ __forceinline__ bool list_add_hi(const OParams &p, int a, int b, int g, int lane) {
    int off = p.seg_off[a];
    const int n = p.seg_len[a];
    int pos = n, at = -1;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int i = c0 + lane;
        const int bb = i < n ? p.eb[off + i] : 0x7FFFFFFF;
        const unsigned eq = __ballot_sync(0xFFFFFFFFu, bb == b);
        if (eq) {
            at = c0 + __ffs(eq) - 1;
            break;
        }
        const unsigned gt = __ballot_sync(0xFFFFFFFFu, bb > b);
        if (gt) {
            pos = c0 + __ffs(gt) - 1;
            break;
        }
    }
    if (at >= 0) {
        if (lane == 0) p.ehi[off + at] += g;
        return true;
    }
    const int cap = p.seg_cap[a];
    if (n == cap) {  // move to a slot of 2 cap entries
        long long o2 = 0;
        if (lane == 0) o2 = (long long)atomicAdd(&p.ctl->arena_top, 2u * (unsigned)cap);
        o2 = __shfl_sync(0xFFFFFFFFu, o2, 0);
        const long long base = (long long)p.nA * kListSlot + o2;
        if (base + 2ll * cap > p.list_cap) {
            if (lane == 0) record_error(&p.ctl->head, PR_ERR_CAPACITY);
            return false;
        }
        for (int i = lane; i < n; i += 32) {
            p.eb[base + i] = p.eb[off + i];
            p.elo[base + i] = p.elo[off + i];
            p.ehi[base + i] = p.ehi[off + i];
        }
        __syncwarp();
        off = (int)base;
        if (lane == 0) {
            p.seg_off[a] = off;
            p.seg_cap[a] = 2 * cap;
        }
    }
    // entries pos .. n - 1 move up by one, the last chunk first (every lane
    // reads its entry before any lane of the warp writes)
    for (int top = n - 1; top >= pos; top -= 32) {
        const int i = top - lane;
        const bool act = i >= pos;
        int vb = 0, vl = 0, vh = 0;
        if (act) {
            vb = p.eb[off + i];
            vl = p.elo[off + i];
            vh = p.ehi[off + i];
        }
        __syncwarp();
        if (act) {
            p.eb[off + i + 1] = vb;
            p.elo[off + i + 1] = vl;
            p.ehi[off + i + 1] = vh;
        }
        __syncwarp();
    }
    if (lane == 0) {
        p.eb[off + pos] = b;
        p.elo[off + pos] = 0;
        p.ehi[off + pos] = g;
        p.seg_len[a] = n + 1;
    }
    return true;
}

// Step (III a) on a's list when its clusters shift up: the lo counts are all
// zero (the lo cluster ran out), every hi count becomes the lo count, and
// entries left with no copies are dropped (the order is kept).
__device__ __forceinline__ void list_shift(const OParams &p, int a, int lane) {
    const int off = p.seg_off[a], n = p.seg_len[a];
    int w = 0;
    bool bad = false;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int i = c0 + lane;
        int bb = 0, hh = 0;
        if (i < n) {
            bb = p.eb[off + i];
            hh = p.ehi[off + i];
            bad |= p.elo[off + i] != 0;
        }
        const unsigned keep = __ballot_sync(0xFFFFFFFFu, hh > 0);
        __syncwarp();
        if (hh > 0) {
            const int k = off + w + __popc(keep & ((1u << lane) - 1));
            p.eb[k] = bb;
            p.elo[k] = hh;
            p.ehi[k] = 0;
        }
        w += __popc(keep);
        __syncwarp();
    }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) record_error(&p.ctl->head, PR_ERR_INTERNAL);
    if (lane == 0) p.seg_len[a] = w;
}

// The demands of one wave of the grid, CTA-minor: thread t of CTA c takes
// demand c + t * G, so every CTA gets about n_dem / G of them.
__device__ __forceinline__ int wave_demand(int base, unsigned G) {
    return base + (int)(threadIdx.x * G + blockIdx.x);
}

// Grant step: thread per demand a that received a proposal in round R; its
// lowest proposer b takes g = min(r_b, avail_a) copies.  The grants go on a
// CTA list; after a CTA barrier each warp takes one listed grant: if a's
// copies are matched (kmin_a >= 1) it evicts g of them (step II), then it
// adds b's g copies to a's list.  Every a has one winner and touches only its
// own list, and the counts other grants also touch (f) change by atomics, so
// the order of the grants does not matter.
__device__ __forceinline__ void ot_grant(const OParams &p, unsigned R) {
    __shared__ int gl_a[kOtThreads], gl_b[kOtThreads], gl_g[kOtThreads];
    __shared__ int n_gl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned G = gridDim.x;
    for (int base = 0; base < p.nA; base += (int)(G * blockDim.x)) {
        if (threadIdx.x == 0) n_gl = 0;
        __syncthreads();
        const int a = wave_demand(base, G);
        if (a < p.nA) {
            // the column's word and the winner's remaining copies were written
            // by other CTAs: coherent loads (L2), never a line this SM's L1
            // kept from an earlier round
            const unsigned long long w = ld_relaxed_u64(p.prop + a);
            if (tag_of(w) == R) {
                const int b = row_of(w);
                // the values a winner needs, loaded at once (only a's winner
                // writes them in this step)
                const int av = p.avail[a];
                const int rb = ld_relaxed_s32(p.r + b);
                const int km = p.kmin[a];
                const int g = rb < av ? rb : av;
                p.avail[a] = av - g;
                p.r[b] = rb - g;
                if (rb - g == 0) atomicAnd(p.flag + b, ~kFlagSearching);
                p.clo[a] -= g;
                p.chi[a] += g;
                p.granted[a] = 1;
                atomicSub(p.f + b, g);
                if (g > 0) {
                    const int k = atomicAdd(&n_gl, 1);
                    gl_a[k] = a;
                    gl_b[k] = b;
                    gl_g[k] = km >= 1 ? -g : g;  // negative: matched copies are taken
                }
            }
        }
        __syncthreads();
        for (int e = warp; e < n_gl; e += nw) {
            const int ga = gl_a[e], gg = gl_g[e];
            if (gg < 0) list_evict(p, ga, -gg, lane);
            __syncwarp();
            list_add_hi(p, ga, gl_b[e], gg < 0 ? -gg : gg, lane);
        }
        __syncthreads();
    }
}

template <class CB>
__device__ __forceinline__ void ot_phase_end(const OParams &p) {
    __shared__ int sh_a[kOtThreads];
    __shared__ int n_sh;
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned G = gridDim.x;
    for (int b = t0; b < p.nB; b += stride)
        if ((ld_relaxed_s32(p.flag + b) & kFlagInBp) && ld_relaxed_s32(p.r + b) > 0) p.F[b] += 1;  // step (III b)
    for (int base = 0; base < p.nA; base += (int)(G * blockDim.x)) {
        if (threadIdx.x == 0) n_sh = 0;
        __syncthreads();
        const int a = wave_demand(base, G);
        if (a < p.nA && p.granted[a]) {
            p.granted[a] = 0;
            if (p.clo[a] == 0 && p.chi[a] > 0) {  // step (III a): clusters shift up
                const int k = p.kmin[a] + 1;
                p.kmin[a] = k;
                static_cast<CB *>(p.key)[a] = (CB)k;  // bytes: k <= floor(1/eps) + 2 <= 254
                p.clo[a] = p.chi[a];
                p.chi[a] = 0;
                sh_a[atomicAdd(&n_sh, 1)] = a;
            }
            p.avail[a] = p.clo[a];
        }
        __syncthreads();
        for (int e = warp; e < n_sh; e += nw) list_shift(p, sh_a[e], lane);
        __syncthreads();
    }
}

// Every phase and round of Sec. 4's cluster form in one cooperative launch;
// grid barriers with summed payloads stand between the steps, so the host
// reads nothing until the loop is over.  The stop rule is Sec. 3.3 on the
// copy instance: T = floor(eps * S), S the total supply copies, the phase cap
// S (2K + 3) / (T + 1) + 1 with K = floor(1/eps).
template <class CB, bool F7>
__global__ void __launch_bounds__(kOtThreads, 4) k_ot_loop(OParams p, double eps, long long spin_limit) {
    OCtl *c = p.ctl;
    // invalid masses or costs (recorded by the earlier kernels of the solve):
    // the copy counts are not all written, so no loop runs (every CTA reads
    // the same value)
    if (ld_relaxed_s32(&c->head.err) != 0) return;
    const unsigned G = gridDim.x;
    unsigned gen = 0;
    unsigned long long sum = 0;
    unsigned long long s_loc = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < p.nB; b += gridDim.x * blockDim.x)
        s_loc += (unsigned long long)p.S[b];
    s_loc = cta_sum(s_loc);
    if (!grid_sum_barrier(c->bar, &c->head, gen, G, spin_limit, s_loc, sum)) return;
    const long long S_total = (long long)sum;
    const long long T = (long long)floor(eps * (double)S_total);
    const long long K = (long long)floor(1.0 / eps);
    const long long cap = (S_total * (2 * K + 3)) / (T + 1) + 1;
    long long phases = 0, rounds = 0;
    unsigned R = 0;
    unsigned long long bytes = 0;
    for (;;) {
        const unsigned long long nf = cta_sum(ot_phase_start(p));
        if (!grid_sum_barrier(c->bar, &c->head, gen, G, spin_limit, nf, sum)) return;
        const long long nfree = (long long)sum;
        if (nfree <= T || phases >= cap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                c->free_at_stop = nfree;
                c->threshold = T;
                if (nfree > T) record_error(&c->head, PR_ERR_NO_CONVERGENCE);
            }
            break;
        }
        ++phases;
        // Every round grants some column's lowest proposer g > 0 copies,
        // which either places all of b's remaining copies (at most |B'|
        // times a phase) or uses up a's available copies (at most n_dem
        // times): a phase has at most n_sup + n_dem rounds with a proposal.
        long long phase_rounds = 0;
        for (;;) {
            ++R;
            if (++phase_rounds > (long long)p.nB + p.nA + 1) {
                if (blockIdx.x == 0 && threadIdx.x == 0) record_error(&c->head, PR_ERR_INTERNAL);
                return;
            }
            const unsigned long long np = cta_sum(ot_propose<CB, F7>(p, R, bytes));
            if (!grid_sum_barrier(c->bar, &c->head, gen, G, spin_limit, np, sum)) return;
            if (sum == 0) break;
            ++rounds;
            ot_grant(p, R);
            if (!grid_sum_barrier(c->bar, &c->head, gen, G, spin_limit, 0, sum)) return;
        }
        ot_phase_end<CB>(p);
        if (!grid_sum_barrier(c->bar, &c->head, gen, G, spin_limit, 0, sum)) return;
    }
    const unsigned long long cb = cta_sum(bytes);
    if (threadIdx.x == 0 && cb) atomicAdd((unsigned long long *)&c->bytes, cb);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->phases = phases;
        c->rounds = rounds;
    }
}

// ---------------------------------------------------------------------------
// Plan and fix-up
// ---------------------------------------------------------------------------
struct FixParams {
    OParams o;
    const double *nu, *mu;
    double theta;
    int *nnz_a, *off_a, *trim_b;
    double *trim_t, *q, *rres;
    int *cnt_b, *off_b, *bsort_a;
    int *nw_b, *nw_a;
    double *nw_t;
    unsigned long long *nw_pr, *nw_pq;  // inclusive prefix sums of the residual units
    int *plan_row, *plan_col;
    double *plan_mass;
    long long plan_cap;
};

// Warp per demand a: nonzero count, the trim of its highest supplier, and the
// remaining capacity q_a = max(0, mu_a - received), sums in ascending b (the
// order of a's list).
__global__ void __launch_bounds__(kOtThreads) k_fix_demand(FixParams fp) {
    const OParams &p = fp.o;
    if (ld_relaxed_s32(&p.ctl->head.err) != 0) return;
    const int lane = threadIdx.x & 31;
    const int warp_g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int a = warp_g; a < p.nA; a += nwarps) {
        const int off = p.seg_off[a], n = p.seg_len[a];
        int nnz = 0, last = -1;
        double recv = 0.0, before_last = 0.0, m_last = 0.0;
        for (int c0 = 0; c0 < n; c0 += 32) {
            const int i = c0 + lane;
            const int c = i < n ? p.elo[off + i] + p.ehi[off + i] : 0;
            const int bb = i < n ? p.eb[off + i] : 0;
            const unsigned nz = __ballot_sync(0xFFFFFFFFu, c != 0);
            if (!nz) continue;
            nnz += __popc(nz);
            const double m = c ? __ddiv_rn((double)c, fp.theta) : 0.0;
            // lane order = ascending b: fold the chunk's masses in that order
            for (unsigned w = nz; w; w &= w - 1) {
                const int L = __ffs(w) - 1;
                const double mi = __shfl_sync(0xFFFFFFFFu, m, L);
                before_last = recv;
                m_last = mi;
                recv = __dadd_rn(recv, mi);
                last = __shfl_sync(0xFFFFFFFFu, bb, L);
            }
        }
        if (lane == 0) {
            fp.nnz_a[a] = nnz;
            const double excess = __dsub_rn(recv, fp.mu[a]);
            int tb = -1;
            double tt = 0.0, r2 = recv;
            if (excess > 0.0 && last >= 0) {
                // every positive mass is >= 1/theta > excess: one trim, on the
                // highest supplier, which is also the last term of the sum
                tb = last;
                tt = m_last < excess ? m_last : excess;
                r2 = __dadd_rn(before_last, __dsub_rn(m_last, tt));
            }
            fp.trim_b[a] = tb;
            fp.trim_t[a] = tt;
            const double qa = __dsub_rn(fp.mu[a], r2);
            fp.q[a] = qa < 0.0 ? 0.0 : qa;
        }
    }
}

// One CTA: exclusive prefix sums of n counts (out[n] = total); each thread
// takes four consecutive counts per step.
__global__ void k_prefix(const int *cnt, int n, int *out) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 4 * blockDim.x) {
        const int i0 = base + 4 * threadIdx.x;
        int v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = i0 + e < n ? cnt[i0 + e] : 0;
        const int own = v[0] + v[1] + v[2] + v[3];
        int x = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const int w = lane < nw ? warp_tot[lane] : 0;
            int z = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, z, o);
                if (lane >= o) z += y;
            }
            if (lane < nw) warp_tot[lane] = z - w;
        }
        __syncthreads();
        int run = carry + warp_tot[warp] + x - own;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (i0 + e < n) out[i0 + e] = run;
            run += v[e];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += warp_tot[warp] + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

// Warp per demand a: write a's plan entries (b ascending, the order of a's
// list) at off_a[a]; count the entries of every supply row.  When the matched
// entries alone exceed plan_cap, PR_ERR_CAPACITY is recorded with their
// count in plan_nnz, and the kernels after this one return at once.
__global__ void __launch_bounds__(kOtThreads) k_fix_write(FixParams fp, int64_t *plan_nnz) {
    const OParams &p = fp.o;
    if (ld_relaxed_s32(&p.ctl->head.err) != 0) return;
    const int total = fp.off_a[p.nA];
    if (total > fp.plan_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *plan_nnz = total;
            record_error(&p.ctl->head, PR_ERR_CAPACITY);
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const int warp_g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int a = warp_g; a < p.nA; a += nwarps) {
        const int off = p.seg_off[a], n = p.seg_len[a];
        const int tb = fp.trim_b[a];
        int k = fp.off_a[a];
        for (int c0 = 0; c0 < n; c0 += 32) {
            const int i = c0 + lane;
            const int c = i < n ? p.elo[off + i] + p.ehi[off + i] : 0;
            const unsigned nz = __ballot_sync(0xFFFFFFFFu, c != 0);
            if (c) {
                const int b = p.eb[off + i];
                double m = __ddiv_rn((double)c, fp.theta);
                if (b == tb) m = __dsub_rn(m, fp.trim_t[a]);
                const int kk = k + __popc(nz & ((1u << lane) - 1));
                fp.plan_row[kk] = b;
                fp.plan_col[kk] = a;
                fp.plan_mass[kk] = m;
                atomicAdd(fp.cnt_b + b, 1);
            }
            k += __popc(nz);
        }
    }
}

// Thread per entry: scatter the entry index into its supply row's segment.
__global__ void k_fix_bscatter(FixParams fp, int *fill) {
    if (ld_relaxed_s32(&fp.o.ctl->head.err) != 0) return;
    const int nnz = fp.off_a[fp.o.nA];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
        const int b = fp.plan_row[k];
        fp.bsort_a[fp.off_b[b] + atomicAdd(fill + b, 1)] = k;
    }
}

// Thread per supply b: its entries in ascending a (insertion sort of the
// row's small segment), then rres_b = max(0, nu_b - sent_b).
__global__ void k_fix_supply(FixParams fp) {
    const OParams &p = fp.o;
    if (ld_relaxed_s32(&fp.o.ctl->head.err) != 0) return;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < p.nB; b += gridDim.x * blockDim.x) {
        const int s = fp.off_b[b], e = fp.off_b[b + 1];
        int *seg = fp.bsort_a + s;
        for (int i = 1; i < e - s; ++i) {
            const int v = seg[i];
            const int av = fp.plan_col[v];
            int j = i - 1;
            while (j >= 0 && fp.plan_col[seg[j]] > av) {
                seg[j + 1] = seg[j];
                --j;
            }
            seg[j + 1] = v;
        }
        double sent = 0.0;
        for (int i = 0; i < e - s; ++i) sent = __dadd_rn(sent, fp.plan_mass[seg[i]]);
        const double rr = __dsub_rn(fp.nu[b], sent);
        fp.rres[b] = rr < 0.0 ? 0.0 : rr;
    }
}

// A residual in whole units of 2^-62, rounded down (the product is exact;
// residuals are below 2, so the units are below 2^63).
__device__ __forceinline__ unsigned long long nw_units(double r) {
    return r > 0.0 ? __double2ull_rz(__dmul_rn(r, 0x1p62)) : 0ull;
}

// How many of P[0..n) (non-decreasing) are <= v, and are < v.
__device__ __forceinline__ int nw_count_le(const unsigned long long *P, int n, unsigned long long v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (P[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int nw_count_lt(const unsigned long long *P, int n, unsigned long long v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (P[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Two CTAs: inclusive prefix sums of the residual units, supplies (CTA 0)
// and demands (CTA 1).  Each thread sums one contiguous run, one scan over
// the threads gives its offset, then the run is written.
__global__ void __launch_bounds__(1024) k_nw_prefix(FixParams fp) {
    if (ld_relaxed_s32(&fp.o.ctl->head.err) != 0) return;
    __shared__ unsigned long long warp_off[32];
    const bool dem = blockIdx.x == 1;
    const double *x = dem ? fp.q : fp.rres;
    const int n = dem ? fp.o.nA : fp.o.nB;
    unsigned long long *P = dem ? fp.nw_pq : fp.nw_pr;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    unsigned long long own = 0;
    for (int k = lo; k < hi; ++k) own += nw_units(x[k]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long inc = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_off[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = lane < nw ? warp_off[lane] : 0;
        unsigned long long z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < nw) warp_off[lane] = z - w;
    }
    __syncthreads();
    unsigned long long run = warp_off[warp] + inc - own;
    for (int k = lo; k < hi; ++k) {
        run += nw_units(x[k]);
        P[k] = run;
    }
}

// Thread per supply and per demand: the start s of its run of units (the
// exclusive prefix sum) and its place in the merged order of all starts
// (supplies before demands on equal starts).  An allocation starts at s if
// the run is not empty and s is below cap = min(totals), except a demand
// whose run starts where a non-empty supply run starts: that allocation is
// the supply's.  flag[place] marks the allocation; the merged order is the
// serial walk's order.
__global__ void k_nw_flags(FixParams fp, int *flag, int *place) {
    if (ld_relaxed_s32(&fp.o.ctl->head.err) != 0) return;
    const int nB = fp.o.nB, nA = fp.o.nA;
    const unsigned long long *Pr = fp.nw_pr, *Pq = fp.nw_pq;
    const unsigned long long cap = Pr[nB - 1] < Pq[nA - 1] ? Pr[nB - 1] : Pq[nA - 1];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nB + nA; k += gridDim.x * blockDim.x) {
        int m, f = 0;
        if (k < nB) {
            const unsigned long long s = k ? Pr[k - 1] : 0ull;
            // demands starting below s: demand 0 (start 0) and every j >= 1 with Pq[j-1] < s
            m = k + (s > 0 ? 1 + nw_count_lt(Pq, nA - 1, s) : 0);
            f = Pr[k] > s && s < cap;
        } else {
            const int j = k - nB;
            const unsigned long long s = j ? Pq[j - 1] : 0ull;
            // supplies starting at or below s: supply 0 and every i >= 1 with Pr[i-1] <= s
            m = j + 1 + nw_count_le(Pr, nB - 1, s);
            if (Pq[j] > s && s < cap) {
                const int i = nw_count_le(Pr, nB, s);  // Pr[i] > s, as s < Pr[nB - 1]
                f = (i ? Pr[i - 1] : 0ull) != s;
            }
        }
        flag[m] = f;
        place[k] = m;
    }
}

// Thread per flagged start: the allocation (b, a, amount) that begins there,
// written at its rank among the flagged starts.  A supply start s lies in
// the demand run j with Pq[j-1] <= s < Pq[j], a demand start in the supply
// run i likewise; the allocation ends at min(Pr[i], Pq[j]).
__global__ void k_nw_write(FixParams fp, const int *flag, const int *place, const int *off, OCtl *ctl) {
    if (ld_relaxed_s32(&fp.o.ctl->head.err) != 0) return;
    const int nB = fp.o.nB, nA = fp.o.nA;
    const unsigned long long *Pr = fp.nw_pr, *Pq = fp.nw_pq;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nB + nA; k += gridDim.x * blockDim.x) {
        const int m = place[k];
        if (!flag[m]) continue;
        int i, j;
        unsigned long long s;
        if (k < nB) {
            i = k;
            s = i ? Pr[i - 1] : 0ull;
            j = nw_count_le(Pq, nA, s);
        } else {
            j = k - nB;
            s = j ? Pq[j - 1] : 0ull;
            i = nw_count_le(Pr, nB, s);
        }
        const unsigned long long e = Pr[i] < Pq[j] ? Pr[i] : Pq[j];
        const int o = off[m];
        fp.nw_b[o] = i;
        fp.nw_a[o] = j;
        fp.nw_t[o] = __dmul_rn(__ull2double_rn(e - s), 0x1p-62);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->n_nw = off[nB + nA];
}

// Thread per north-west allocation: add it to the matched entry of (b, a)
// (binary search in a's segment, ascending b), or flag it as a new entry.
__global__ void k_fix_merge(FixParams fp, OCtl *ctl, int *flag) {
    if (ld_relaxed_s32(&fp.o.ctl->head.err) != 0) return;
    const int n = ctl->n_nw;
    const int total = fp.o.nB + fp.o.nA;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        int fl = 0;
        if (k < n) {
            const int b = fp.nw_b[k], a = fp.nw_a[k];
            int lo = fp.off_a[a], hi = fp.off_a[a + 1] - 1, at = -1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int bm = fp.plan_row[mid];
                if (bm == b) {
                    at = mid;
                    break;
                }
                if (bm < b) lo = mid + 1;
                else hi = mid - 1;
            }
            if (at >= 0) fp.plan_mass[at] = __dadd_rn(fp.plan_mass[at], fp.nw_t[k]);
            else fl = 1;
        }
        flag[k] = fl;
    }
}

// New pairs go after the matched entries, in north-west order.  A plan that
// then exceeds plan_cap records PR_ERR_CAPACITY with its size in plan_nnz.
__global__ void k_fix_append(FixParams fp, OCtl *ctl, const int *flag, const int *off, int64_t *plan_nnz) {
    if (ld_relaxed_s32(&fp.o.ctl->head.err) != 0) return;
    const int n = ctl->n_nw;
    const int nnz = fp.off_a[fp.o.nA];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (!flag[k]) continue;
        const long long pos = (long long)nnz + off[k];
        if (pos < fp.plan_cap) {
            fp.plan_row[pos] = fp.nw_b[k];
            fp.plan_col[pos] = fp.nw_a[k];
            fp.plan_mass[pos] = fp.nw_t[k];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int extra = off[fp.o.nB + fp.o.nA];
        ctl->n_extra = extra;
        if ((long long)nnz + extra > fp.plan_cap) {
            *plan_nnz = (long long)nnz + extra;
            record_error(&ctl->head, PR_ERR_CAPACITY);
        }
    }
}

// cost = sum mass * c over the plan in a fixed order: kCostCtas CTAs each
// take one contiguous share of the entries (a fixed tree inside the CTA); the
// CTA that finishes last adds the kCostCtas partial sums in CTA order.
template <class T>
__global__ void __launch_bounds__(256)
k_fix_cost(FixParams fp, const T *C, long long ldc, OCtl *ctl, int64_t *plan_nnz, double *cost) {
    __shared__ double part[256];
    __shared__ bool last;
    if (ld_relaxed_s32(&fp.o.ctl->head.err) != 0) return;
    const int nnz = fp.off_a[fp.o.nA] + ctl->n_extra;
    const int lim = nnz < fp.plan_cap ? nnz : (int)fp.plan_cap;
    const int per = (lim + (int)gridDim.x - 1) / (int)gridDim.x;
    const int k0 = blockIdx.x * per, k1 = min(lim, k0 + per);
    double acc = 0.0;
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x)
        acc = __dadd_rn(acc, __dmul_rn(fp.plan_mass[k], (double)C[(long long)fp.plan_row[k] * ldc + fp.plan_col[k]]));
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ctl->cost_part[blockIdx.x] = part[0];
        __threadfence();
        last = atomicAdd(&ctl->cost_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const volatile double *cp = ctl->cost_part;
        double s = 0.0;
        for (unsigned c = 0; c < gridDim.x; ++c) s = __dadd_rn(s, cp[c]);
        *cost = s;
        *plan_nnz = nnz;
    }
}

__global__ void k_ot_duals(OParams p, int *y_sup, int *dem_kmin, int *dem_lo, int *dem_hi) {
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int b = t0; b < p.nB; b += stride) y_sup[b] = p.F[b];
    for (int a = t0; a < p.nA; a += stride) {
        dem_kmin[a] = p.kmin[a];
        dem_lo[a] = p.clo[a];
        dem_hi[a] = p.chi[a];
    }
}

__global__ void k_zero_int(int *x, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0;
}

}  // namespace
}  // namespace prot

using namespace prot;

extern "C" size_t pr_ot_workspace(int32_t n_sup, int32_t n_dem) {
    if (n_sup < 1 || n_dem < 1 || n_sup > (1 << 24) || n_dem > (1 << 24)) return 0;
    if ((size_t)n_sup * (size_t)n_dem > ((size_t)1 << 31) - 1) return 0;
    return make_olayout(n_sup, n_dem).total;
}

extern "C" pr_status pr_ot(const void *C, pr_dtype dt, int64_t ldc, int32_t n_sup, int32_t n_dem,
                           const double *supply, const double *demand, double eps,
                           int64_t plan_cap, int32_t *plan_row, int32_t *plan_col,
                           double *plan_mass, int64_t *plan_nnz, int32_t *y_sup,
                           int32_t *dem_kmin, int32_t *dem_lo, int32_t *dem_hi, double *cost,
                           pr_stats *stats, void *ws, size_t ws_bytes, void *stream) {
    if (!C || !supply || !demand || !plan_row || !plan_col || !plan_mass || !plan_nnz || !y_sup ||
        !dem_kmin || !dem_lo || !dem_hi || !cost)
        return fail(PR_ERR_INVALID, "pr_ot: NULL pointer argument");
    if (dt != PR_F32 && dt != PR_F64) return fail(PR_ERR_INVALID, "pr_ot: bad dtype");
    if (n_sup < 1 || n_dem < 1 || n_sup > (1 << 24) || n_dem > (1 << 24) ||
        (size_t)n_sup * (size_t)n_dem > ((size_t)1 << 31) - 1)
        return fail(PR_ERR_INVALID, "pr_ot: need 1 <= n_sup, n_dem and n_sup * n_dem < 2^31");
    if (ldc < n_dem) return fail(PR_ERR_INVALID, "pr_ot: ldc < n_dem");
    if (!(eps > 0.0 && eps < 1.0) || floor(1.0 / eps) > 32766.0)
        return fail(PR_ERR_INVALID, "pr_ot: need 0 < eps < 1 and floor(1/eps) <= 32766");
    if (plan_cap < 1) return fail(PR_ERR_INVALID, "pr_ot: plan_cap must be >= 1");
    const OLayout L = make_olayout(n_sup, n_dem);
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < L.total)
        return fail(PR_ERR_WORKSPACE, "pr_ot: workspace NULL, not 256-byte aligned or < %zu bytes", L.total);
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    const int nB = n_sup, nA = n_dem;
    const int n = nB > nA ? nB : nA;
    const double theta = (4.0 * (double)n) / eps;

    OParams p;
    p.ctl = (OCtl *)(w + L.ctl);
    p.cb = w + L.cb;
    p.key = w + L.key;
    p.S = (int *)(w + L.S);
    p.D = (int *)(w + L.D);
    p.F = (int *)(w + L.F);
    p.f = (int *)(w + L.f);
    p.r = (int *)(w + L.r);
    p.ptr = (int *)(w + L.ptr);
    p.flag = (int *)(w + L.flag);
    p.kmin = (int *)(w + L.kmin);
    p.clo = (int *)(w + L.clo);
    p.chi = (int *)(w + L.chi);
    p.avail = (int *)(w + L.avail);
    p.granted = (int *)(w + L.granted);
    p.prop = (unsigned long long *)(w + L.prop);
    p.eb = (int *)(w + L.eb);
    p.elo = (int *)(w + L.elo);
    p.ehi = (int *)(w + L.ehi);
    p.seg_off = (int *)(w + L.seg_off);
    p.seg_cap = (int *)(w + L.seg_cap);
    p.seg_len = (int *)(w + L.seg_len);
    p.list_cap = L.list_cap;
    p.nB = nB;
    p.nA = nA;
    p.ldq = L.ldq;

    const DeviceInfo &di = device_info();
    const int g1 = di.sms * 4;
    k_ot_ctl_init<<<1, 1, 0, st>>>(p.ctl);
    PR_CUDA(cudaGetLastError());
    k_ot_counts<<<g1, 256, 0, st>>>(supply, demand, nB, nA, theta, p.S, p.D, p.ctl);
    PR_CUDA(cudaGetLastError());
    // bytes for the rounded costs and keys when every cbar and key fits one
    // (floor(1/eps) <= 252, as in pr_assign)
    const bool cb8 = floor(1.0 / eps) <= 252.0;
    if (cb8) k_ot_init<uint8_t><<<g1 * 4, 256, 0, st>>>(p);
    else k_ot_init<uint16_t><<<g1 * 4, 256, 0, st>>>(p);
    PR_CUDA(cudaGetLastError());
    {
        const long long groups = (long long)nB * (L.ldq >> 3);
        const long long want = groups / 256 + 1;
        const int qgrid = (int)std::min<long long>(want, (long long)di.sms * 16);
        void *cbw = const_cast<void *>(p.cb);
        if (dt == PR_F64 && cb8)
            launch_quantise<double, uint8_t>((const double *)C, ldc, nB, nA, L.ldq, eps, (uint8_t *)cbw,
                                             &p.ctl->head, qgrid, st);
        else if (dt == PR_F64)
            launch_quantise<double, uint16_t>((const double *)C, ldc, nB, nA, L.ldq, eps, (uint16_t *)cbw,
                                              &p.ctl->head, qgrid, st);
        else if (cb8)
            launch_quantise<float, uint8_t>((const float *)C, ldc, nB, nA, L.ldq, eps, (uint8_t *)cbw,
                                            &p.ctl->head, qgrid, st);
        else
            launch_quantise<float, uint16_t>((const float *)C, ldc, nB, nA, L.ldq, eps, (uint16_t *)cbw,
                                             &p.ctl->head, qgrid, st);
        PR_CUDA(cudaGetLastError());
    }
    const int gw = di.sms * 8;  // warps-per-row kernels of the fix-up: grid of 256-thread CTAs
    {
        // the phase loop: one cooperative launch, as many CTAs as fit (at
        // most 1023, the barrier's arrival field)
        const bool f7 = floor(1.0 / eps) <= 125.0;
        const void *loop = !cb8 ? (const void *)k_ot_loop<uint16_t, false>
                                : f7 ? (const void *)k_ot_loop<uint8_t, true> : (const void *)k_ot_loop<uint8_t, false>;
        int per_sm = 0;
        PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, loop, kOtThreads, 0));
        if (per_sm < 1) return fail(PR_ERR_INVALID, "pr_ot: loop kernel does not fit on an SM");
        const int grid = std::min(di.sms * per_sm, 1023);
        const long long limit = spin_limit_cycles();
        void *args[] = {(void *)&p, (void *)&eps, (void *)&limit};
        PR_CUDA(cudaLaunchCooperativeKernel(loop, dim3(grid), dim3(kOtThreads), args, 0, st));
    }
    // plan and fix-up
    FixParams fp;
    fp.o = p;
    fp.nu = supply;
    fp.mu = demand;
    fp.theta = theta;
    fp.nnz_a = (int *)(w + L.nnz_a);
    fp.off_a = (int *)(w + L.off_a);
    fp.trim_b = (int *)(w + L.trim_b);
    fp.trim_t = (double *)(w + L.trim_t);
    fp.q = (double *)(w + L.q);
    fp.rres = (double *)(w + L.rres);
    fp.cnt_b = (int *)(w + L.cnt_b);
    fp.off_b = (int *)(w + L.off_b);
    fp.bsort_a = (int *)(w + L.bsort_a);
    fp.nw_b = (int *)(w + L.nw_b);
    fp.nw_a = (int *)(w + L.nw_a);
    fp.nw_t = (double *)(w + L.nw_t);
    fp.nw_pr = (unsigned long long *)(w + L.nw_pr);
    fp.nw_pq = (unsigned long long *)(w + L.nw_pq);
    fp.plan_row = plan_row;
    fp.plan_col = plan_col;
    fp.plan_mass = plan_mass;
    fp.plan_cap = plan_cap;
    k_fix_demand<<<gw, kOtThreads, 0, st>>>(fp);
    PR_CUDA(cudaGetLastError());
    k_prefix<<<1, 1024, 0, st>>>(fp.nnz_a, nA, fp.off_a);
    PR_CUDA(cudaGetLastError());
    k_zero_int<<<g1, 256, 0, st>>>(fp.cnt_b, nB);
    k_fix_write<<<gw, kOtThreads, 0, st>>>(fp, plan_nnz);
    PR_CUDA(cudaGetLastError());
    k_prefix<<<1, 1024, 0, st>>>(fp.cnt_b, nB, fp.off_b);
    k_zero_int<<<g1, 256, 0, st>>>(fp.cnt_b, nB);
    k_fix_bscatter<<<g1, 256, 0, st>>>(fp, fp.cnt_b);
    k_fix_supply<<<(nB + 255) / 256, 256, 0, st>>>(fp);
    PR_CUDA(cudaGetLastError());
    {
        // the north-west allocations; their flags and ranks use the arrays
        // that the merge below then reuses
        int *flag = (int *)(w + L.nw_flag), *off = (int *)(w + L.nw_off), *place = (int *)(w + L.nw_pos);
        k_nw_prefix<<<2, 1024, 0, st>>>(fp);
        k_nw_flags<<<g1, 256, 0, st>>>(fp, flag, place);
        k_prefix<<<1, 1024, 0, st>>>(flag, nB + nA, off);
        k_nw_write<<<g1, 256, 0, st>>>(fp, flag, place, off, p.ctl);
        PR_CUDA(cudaGetLastError());
    }
    {
        int *flag = (int *)(w + L.nw_flag), *off = (int *)(w + L.nw_off);
        k_fix_merge<<<g1, 256, 0, st>>>(fp, p.ctl, flag);
        PR_CUDA(cudaGetLastError());
        k_prefix<<<1, 1024, 0, st>>>(flag, nB + nA, off);
        k_fix_append<<<g1, 256, 0, st>>>(fp, p.ctl, flag, off, plan_nnz);
        PR_CUDA(cudaGetLastError());
    }
    if (dt == PR_F64)
        k_fix_cost<double><<<kCostCtas, 256, 0, st>>>(fp, (const double *)C, ldc, p.ctl, plan_nnz, cost);
    else
        k_fix_cost<float><<<kCostCtas, 256, 0, st>>>(fp, (const float *)C, ldc, p.ctl, plan_nnz, cost);
    PR_CUDA(cudaGetLastError());
    k_ot_duals<<<g1, 256, 0, st>>>(p, y_sup, dem_kmin, dem_lo, dem_hi);
    PR_CUDA(cudaGetLastError());
    if (!stats) return PR_OK;  // asynchronous: device errors through pr_ws_status
    OCtl h;
    PR_CUDA(cudaMemcpyAsync(&h, p.ctl, sizeof(OCtl), cudaMemcpyDeviceToHost, st));
    PR_CUDA(cudaStreamSynchronize(st));
    stats->phases = h.phases;
    stats->rounds = h.rounds;
    stats->bytes_scanned = h.bytes;
    stats->rows_scanned = 0;
    stats->free_at_stop = (int32_t)h.free_at_stop;
    stats->threshold = (int32_t)h.threshold;
    stats->loop_ctas = 0;
    stats->loop_cluster = 0;
    stats->cells_examined = 0;
    stats->barriers = 0;
    if (h.head.err == PR_ERR_INVALID && (h.mass_units[0] >= (3ull << 31) || h.mass_units[1] >= (3ull << 31)))
        return fail(PR_ERR_INVALID, "pr_ot: the supply and the demand masses must each sum to 1 "
                                    "(a side summing to more than 1.5 is refused)");
    if (h.head.err == PR_ERR_INVALID) return fail(PR_ERR_INVALID, "pr_ot: invalid costs or masses");
    if (h.head.err == PR_ERR_CAPACITY && h.arena_top > (unsigned)L.arena)
        return fail(PR_ERR_CAPACITY, "pr_ot: the per-demand lists need more than the workspace's %lld arena entries",
                    (long long)L.arena);
    if (h.head.err == PR_ERR_CAPACITY)
        return fail(PR_ERR_CAPACITY, "pr_ot: the plan exceeds plan_cap (%lld entries; plan_nnz holds the size)",
                    (long long)plan_cap);
    if (h.head.err) return fail((pr_status)h.head.err, "pr_ot: device reported %s", pr_status_string((pr_status)h.head.err));
    return PR_OK;
}
