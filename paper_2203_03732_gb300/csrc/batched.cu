// batched.cu -- many independent assignment problems in one persistent launch.
//
// Each CTA pulls problems from a queue in longest-first order (LPT on n) and
// runs the whole main routine of Sec. 2.2 on one problem with every piece of
// per-problem state in shared memory: the keys k(A), the proposal words, the
// row duals, the free-row lists and the proposal lists.  Rounds are separated
// by __syncthreads() instead of a grid barrier.  Only the rounded cost rows
// are read from global memory (HBM / L2), one warp per row.
//
// Problem i is square (n_i rows and columns).  Packed layouts:
//   costs   C[c_off_i + b * n_i + a], c_off_i = sum_{j<i} n_j^2 (rows = B)
//   points  XA[(v_off_i + a) * dim + k], XB[(v_off_i + b) * dim + k]
//   vectors row_to_col[v_off_i + b] (a column of problem i), v_off_i = sum_{j<i} n_j
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "prot_internal.cuh"
#include "scan_common.cuh"
#include "quantise.cuh"
#include "points.cuh"

namespace prot {
namespace {

constexpr int kMaxN = 5000;               // largest problem whose state fits shared memory
constexpr int kRowBits = 13;              // a free-list entry: row | resume column << 13
constexpr int kRowMask = (1 << kRowBits) - 1;
static_assert(kMaxN < (1 << kRowBits), "rows and resume columns must fit 13 bits");
constexpr int kMaxCbarByte = 252;         // byte storage when floor(1/eps) <= 252 (as pr_assign)

struct BDesc {
    long long cb_off;  // element offset of the rounded costs (row stride ldq)
    long long c_off;   // element offset of the cost matrix (matrix source)
    long long cap;     // phase cap
    int n;
    int ldq;
    int v_off;
    int T;
};

struct BCtl {
    WsHead head;
    unsigned queue;
    unsigned pad;
    long long phases;
    long long rounds;
    unsigned long long bytes;
    unsigned long long rows;
};

struct BLayout {
    size_t ctl, desc, order, maxbits, cb, total;
};

BLayout make_blayout(int P, long long cb_elems) {
    BLayout L;
    Carver c;
    L.ctl = c.take<BCtl>(1);
    L.desc = c.take<BDesc>(P);
    L.order = c.take<int>(P);
    L.maxbits = c.take<unsigned>(P);
    L.cb = c.take<uint16_t>((size_t)cb_elems);
    L.total = c.total();
    return L;
}

struct BParams {
    BCtl *ctl;
    const BDesc *desc;
    const int *order;
    const unsigned *maxbits;
    const void *cb;  // uint8_t or uint16_t, as k_bsolve is instantiated
    int nprob;
    int n_max;
    int ldq_max;
    // cost source for the reported costs
    const void *C;
    int dt;  // PR_F32 / PR_F64 (matrix source)
    const float *XA, *XB;
    int dim, squared, points;
    // outputs
    int *row_to_col, *col_to_row, *y_row, *y_col;
    double *costs;
    int64_t *phases;
};

// ---------------------------------------------------------------------------
// Rounding of the packed matrices (Eq. 1, exact).
// ---------------------------------------------------------------------------
// Padding of the stored type: uint16 0x7FFF or, when floor(1/eps) <= 252, byte 0xFF.
template <class CB> constexpr uint32_t kPadOf = sizeof(CB) == 1 ? 0xFFu : (uint32_t)kPadCost;

// Every kernel below takes the rows of all problems in one sweep: warp w takes
// global rows w, w + W, ... (global row r is row r - v_off_i of the problem i
// with v_off_i <= r < v_off_i + n_i, found once per row), and its lanes take
// consecutive columns, so each load instruction of a warp reads one
// contiguous piece of the row and each store writes one contiguous piece of
// the rounded row (padding columns n_i .. ldq_i - 1 included).
__device__ __forceinline__ int problem_of_row(const BDesc *d, int P, int r) {
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].v_off <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Columns per lane in flight per step of the matrix rounding: 2 KiB per warp
// (16 FP32 or 8 FP64 values a lane), 64 KiB per SM at 32 warps, enough to
// cover the load latency at the copy rate (1 KiB per warp reached 3.4 TB/s).
template <class T> constexpr int kRowUnroll = sizeof(T) == 8 ? 8 : 16;
// Columns per lane in flight per step of the points kernels.
constexpr int kPtUnroll = 4;

__device__ __forceinline__ uint32_t quantise_val(double x, const EpsSplit &e) {
    const unsigned long long bits = __double_as_longlong(x);
    return quantise_bits((uint32_t)(bits >> 32), (uint32_t)bits, e);
}
__device__ __forceinline__ uint32_t quantise_val(float x, const EpsSplit &e) {
    return quantise_fbits(__float_as_uint(x), e);
}

// Eq. (1) on the packed matrices, exactly as k_quantise does for one problem.
template <class T, class CB>
__global__ void __launch_bounds__(256, 4) k_bquant_matrix(const T *__restrict__ C, const BDesc *__restrict__ d, int P, int total_rows,
                                EpsSplit e, CB *__restrict__ cb, WsHead *head) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < total_rows; r += nw) {
        const int i = problem_of_row(d, P, r);
        const BDesc D = d[i];
        const int b = r - D.v_off;
        const T *row = C + D.c_off + (long long)b * D.n;
        CB *out = cb + D.cb_off + (long long)b * D.ldq;
        for (int a0 = 0; a0 < D.ldq; a0 += 32 * kRowUnroll<T>) {
            T x[kRowUnroll<T>];
#pragma unroll
            for (int u = 0; u < kRowUnroll<T>; ++u) {
                const int a = a0 + 32 * u + lane;
                x[u] = a < D.n ? __ldg(row + a) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < kRowUnroll<T>; ++u) {
                const int a = a0 + 32 * u + lane;
                if (a >= D.ldq) break;
                uint32_t q = kPadOf<CB>;
                if (a < D.n) {
                    q = quantise_val(x[u], e);
                    if (q == 0xFFFFFFFFu) {
                        bad = true;
                        q = 0;
                    }
                }
                out[a] = (CB)q;
            }
        }
    }
    if (bad) record_error(head, PR_ERR_INVALID);
}

// ---------------------------------------------------------------------------
// Costs from points (points.cuh): c = RN32(d / max d) per problem.
// ---------------------------------------------------------------------------
// d(b, a) from b's coordinates held in registers, in the operation order of
// dist_f32 (ascending k, one IEEE operation at a time); DIM > 0 is the
// dimension known at compile time.
template <int DIM>
__device__ __forceinline__ float dist_regs(const float (&xb)[DIM], const float (&xa)[DIM], int squared) {
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float t = __fsub_rn(xb[k], xa[k]);
        const float sq = __fmul_rn(t, t);
        acc = k == 0 ? sq : __fadd_rn(acc, sq);
    }
    return squared ? acc : __fsqrt_rn(acc);
}

// Largest distance of every problem: a warp's maximum over one row, then one
// atomic per row (non-negative floats order like their bit patterns).  DIM =
// 0: any dimension, one column at a time; DIM > 0: each lane loads the
// coordinates of kPtUnroll columns before it computes.
template <int DIM>
__global__ void k_bpoints_max(const float *__restrict__ XA, const float *__restrict__ XB, int dim,
                              int squared, const BDesc *__restrict__ d, int P, int total_rows,
                              unsigned *maxbits) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < total_rows; r += nw) {
        const int i = problem_of_row(d, P, r);
        const BDesc D = d[i];
        const float *xbp = XB + (long long)r * dim;  // row b of problem i is global row r
        float m = 0.0f;
        if (DIM == 0) {
            for (int a = lane; a < D.n; a += 32)
                m = fmaxf(m, dist_f32(xbp, XA + (long long)(D.v_off + a) * dim, dim, squared));
        } else {
            constexpr int DD = DIM > 0 ? DIM : 1;
            float xb[DD];
#pragma unroll
            for (int k = 0; k < DD; ++k) xb[k] = xbp[k];
            for (int a0 = 0; a0 < D.n; a0 += 32 * kPtUnroll) {
                float xa[kPtUnroll][DD];
#pragma unroll
                for (int u = 0; u < kPtUnroll; ++u) {
                    const int a = a0 + 32 * u + lane;
                    const float *q = XA + (long long)(D.v_off + (a < D.n ? a : 0)) * DD;
#pragma unroll
                    for (int k = 0; k < DD; ++k) xa[u][k] = __ldg(q + k);
                }
#pragma unroll
                for (int u = 0; u < kPtUnroll; ++u)
                    if (a0 + 32 * u + lane < D.n) m = fmaxf(m, dist_regs<DD>(xb, xa[u], squared));
            }
        }
        const unsigned mx = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(m));
        if (lane == 0) atomicMax(maxbits + i, mx);
    }
}

template <int DIM, class CB>
__global__ void k_bpoints_quant(const float *__restrict__ XA, const float *__restrict__ XB, int dim,
                                int squared, const BDesc *__restrict__ d, int P, int total_rows,
                                const unsigned *__restrict__ maxbits, EpsSplit e, CB *__restrict__ cb) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < total_rows; r += nw) {
        const int i = problem_of_row(d, P, r);
        const BDesc D = d[i];
        const int b = r - D.v_off;
        const float M = __uint_as_float(maxbits[i]);
        const float *xbp = XB + (long long)r * dim;
        CB *out = cb + D.cb_off + (long long)b * D.ldq;
        if (DIM == 0) {
            for (int a = lane; a < D.ldq; a += 32) {
                uint32_t q = kPadOf<CB>;
                if (a < D.n) {
                    const float dd = dist_f32(xbp, XA + (long long)(D.v_off + a) * dim, dim, squared);
                    const float c = M > 0.0f ? __fdiv_rn(dd, M) : 0.0f;
                    q = quantise_fbits(__float_as_uint(c), e);
                }
                out[a] = (CB)q;
            }
        } else {
            constexpr int DD = DIM > 0 ? DIM : 1;
            float xb[DD];
#pragma unroll
            for (int k = 0; k < DD; ++k) xb[k] = xbp[k];
            for (int a0 = 0; a0 < D.ldq; a0 += 32 * kPtUnroll) {
                float xa[kPtUnroll][DD];
#pragma unroll
                for (int u = 0; u < kPtUnroll; ++u) {
                    const int a = a0 + 32 * u + lane;
                    const float *q = XA + (long long)(D.v_off + (a < D.n ? a : 0)) * DD;
#pragma unroll
                    for (int k = 0; k < DD; ++k) xa[u][k] = __ldg(q + k);
                }
#pragma unroll
                for (int u = 0; u < kPtUnroll; ++u) {
                    const int a = a0 + 32 * u + lane;
                    if (a >= D.ldq) break;
                    uint32_t q = kPadOf<CB>;
                    if (a < D.n) {
                        const float dd = dist_regs<DD>(xb, xa[u], squared);
                        const float c = M > 0.0f ? __fdiv_rn(dd, M) : 0.0f;
                        q = quantise_fbits(__float_as_uint(c), e);
                    }
                    out[a] = (CB)q;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The per-problem solver.
// ---------------------------------------------------------------------------
struct BShared {
    int nfl[2], nql[2], nwon;
    int had_prop, nonfirst;
    int cur_problem;
    int total;
    int warp_tot[32];
    unsigned long long bytes, rows;
};

// Lowest column a >= start of the row with cbar + k(a) == tgt whose word does
// not carry a tag in [Rps, R) (taken earlier in this phase), or -1.  UNROLL
// 16-byte loads per lane are in flight per step.
template <int UNROLL, class CB, bool F7>
__device__ __forceinline__ int warp_scan_row(const CB *__restrict__ row, const CB *ks,
                                             const unsigned long long *pw, int start, int ldq,
                                             uint32_t tgt, unsigned R, unsigned Rps, int lane,
                                             unsigned long long &bytes) {
    constexpr int W = 16 / (int)sizeof(CB);  // columns per 16-byte load
    constexpr unsigned kAll = W == 16 ? 0xFFFFu : 0xFFu;
    const uint32_t t2 = W == 8 ? (tgt | (tgt << 16)) : tgt * 0x01010101u;
    const bool check_taken = R > Rps;
    for (int c0 = start & ~(W - 1); c0 < ldq; c0 += 32 * W * UNROLL) {
        uint4 cv[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int idx = c0 + u * 32 * W + lane * W;
            cv[u] = idx < ldq ? ld_nc_na_v4(row + idx) : make_uint4(0, 0, 0, 0);
        }
        bytes += sizeof(CB) * (unsigned long long)min(32 * W * UNROLL, ldq - c0);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int idx = c0 + u * 32 * W + lane * W;
            unsigned m = 0;
            if (idx < ldq) {
                const uint4 kv = *reinterpret_cast<const uint4 *>(ks + idx);
                m = W == 8 ? eq_mask(make_uint4(cv[u].x + kv.x, cv[u].y + kv.y, cv[u].z + kv.z, cv[u].w + kv.w), t2)
                           : eq_mask8<F7>(cv[u], kv, t2);
            }
            const int lo = start - idx;
            if (lo > 0) m &= lo >= W ? 0u : (kAll << lo) & kAll;
            for (;;) {
                const unsigned any = __ballot_sync(0xFFFFFFFFu, m != 0);
                if (any == 0) break;
                const int L = __ffs(any) - 1;
                const int a = __shfl_sync(0xFFFFFFFFu, idx + __ffs(m) - 1, L);
                bool taken = false;
                if (check_taken) {
                    const unsigned t = tag_of(pw[a]);
                    taken = t >= Rps && t < R;
                }
                if (!taken) return a;
                if (lane == L) m &= m - 1;
            }
        }
    }
    return -1;
}

__device__ __forceinline__ int block_scan_excl(int flag, BShared &s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, flag);
    const int within = __popc(bal & ((1u << lane) - 1));
    if (lane == 0) s.warp_tot[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
        const int v = lane < nw ? s.warp_tot[lane] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < nw) s.warp_tot[lane] = x - v;
        if (lane == 31) s.total = x;
    }
    __syncthreads();
    const int r = s.warp_tot[warp] + within;
    __syncthreads();
    return r;
}

// F7: floor(1/eps) <= 125, so every sum of a real column's cbar and key
// stays below 256 and the byte pre-test is one plain add (may_match<true>).
template <int THREADS, int UNROLL, class CB, bool F7>
__global__ void __launch_bounds__(THREADS, 1) k_bsolve(BParams p) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ BShared s;
    // region sizes use n_max rounded up to a multiple of 8, so every region
    // (8-byte words, int2 pairs, the uint4-read key copy) starts 16-byte aligned
    const int nmax = (p.n_max + 7) & ~7;
    unsigned long long *pw = reinterpret_cast<unsigned long long *>(dyn);
    int *yb = reinterpret_cast<int *>(pw + nmax);
    int *fl0 = yb + nmax;
    int *fl1 = fl0 + nmax;
    int2 *ql0 = reinterpret_cast<int2 *>(fl1 + nmax);
    int2 *ql1 = ql0 + nmax;
    int *won = reinterpret_cast<int *>(ql1 + nmax);
    CB *ks = reinterpret_cast<CB *>(won + nmax);  // keys in the stored type (bytes: padding 0xFF)
    int *fl[2] = {fl0, fl1};
    int2 *ql[2] = {ql0, ql1};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) s.bytes = s.rows = 0;
    long long my_phases = 0, my_rounds = 0;

    for (;;) {
        if (threadIdx.x == 0) {
            int t = (int)atomicAdd(&p.ctl->queue, 1u);
            if (ld_relaxed_s32(&p.ctl->head.abort)) t = p.nprob;  // stop after an error
            s.cur_problem = t;
        }
        __syncthreads();
        const int t = s.cur_problem;
        __syncthreads();  // every thread has read cur_problem before it changes
        if (t >= p.nprob) break;
        const int pi = p.order[t];
        const BDesc D = p.desc[pi];
        const int n = D.n, ldq = D.ldq;
        const CB *cb = static_cast<const CB *>(p.cb) + D.cb_off;

        // Initialisation (Sec. 2.2): y(b) = eps, y(a) = 0, M empty, B' = B.
        for (int a = threadIdx.x; a < ldq; a += blockDim.x) ks[a] = a < n ? (CB)0 : (CB)(sizeof(CB) == 1 ? 0xFF : kPadKey);
        for (int a = threadIdx.x; a < n; a += blockDim.x) pw[a] = word_of(0, -1);
        for (int b = threadIdx.x; b < n; b += blockDim.x) {
            yb[b] = 1;
            fl0[b] = b;
        }
        if (threadIdx.x == 0) {
            s.nfl[0] = n;
            s.nfl[1] = 0;
        }
        __syncthreads();

        unsigned R = 0;
        long long phases = 0;
        int cur = 0, qcur = 0;
        bool failed = false;
        for (;;) {
            const int nf = s.nfl[cur];
            if (nf <= D.T) break;
            if (phases >= D.cap) {
                failed = true;
                break;
            }
            ++phases;
            const unsigned Rps = R + 1;
            __syncthreads();
            if (threadIdx.x == 0) {
                s.nfl[cur ^ 1] = 0;
                s.nwon = 0;
            }
            bool first = true;
            for (;;) {
                ++R;
                if (threadIdx.x == 0) {
                    s.nql[qcur] = 0;
                    s.had_prop = 0;
                    s.nonfirst = 0;
                }
                __syncthreads();
                const int items = first ? nf : s.nql[qcur ^ 1];
                unsigned long long my_bytes = 0;
                for (int it = warp; it < items; it += nwarps) {
                    int b, start = 0;
                    if (first) {
                        // b, or b | (resume column << 13) for an evicted row
                        const int e = fl[cur][it];
                        b = e & kRowMask;
                        start = e >> kRowBits;
                    } else {
                        const int2 q = ql[qcur ^ 1][it];
                        b = q.x;
                        if (row_of(pw[q.y]) == b) continue;  // won: matched
                        start = q.y + 1;                     // lost: resume after a
                    }
                    const uint32_t tgt = (uint32_t)(yb[b] - 1);
                    const int a = warp_scan_row<UNROLL, CB, F7>(cb + (long long)b * ldq, ks, pw, start, ldq, tgt, R,
                                                            Rps, lane, my_bytes);
                    if (lane == 0) {
                        if (a >= 0) {
                            const unsigned long long old = atomicMax(pw + a, word_of(R, b));
                            if (tag_of(old) < Rps) {
                                // first proposal: a is won this round (step III a
                                // at the phase end), its partner is evicted (II)
                                won[atomicAdd(&s.nwon, 1)] = a;
                                // the evicted row resumes after a: every column
                                // <= a is above its (unchanged) target for good
                                const int partner = row_of(old);
                                if (partner >= 0)
                                    fl[cur ^ 1][atomicAdd(&s.nfl[cur ^ 1], 1)] = partner | ((a + 1) << kRowBits);
                            } else {
                                s.nonfirst = 1;
                            }
                            const int j = atomicAdd(&s.nql[qcur], 1);
                            ql[qcur][j] = make_int2(b, a);
                            s.had_prop = 1;
                        } else {
                            yb[b] += 1;  // step (III b): relabel
                            fl[cur ^ 1][atomicAdd(&s.nfl[cur ^ 1], 1)] = b;
                        }
                    }
                }
                if (lane == 0) {
                    if (my_bytes) atomicAdd(&s.bytes, my_bytes);
                }
                __syncthreads();
                const bool had = s.had_prop != 0, contested = s.nonfirst != 0;
                if (threadIdx.x == 0) s.rows += (unsigned long long)items;
                __syncthreads();
                if (had) ++my_rounds;
                qcur ^= 1;
                first = false;
                if (!contested) break;
            }
            // step (III a): y(a) -= eps for the columns won in this phase
            for (int i = threadIdx.x; i < s.nwon; i += blockDim.x) ks[won[i]] += (CB)1;
            cur ^= 1;
            __syncthreads();
        }
        my_phases += phases;
        if (failed) {
            if (threadIdx.x == 0) record_error(&p.ctl->head, PR_ERR_NO_CONVERGENCE);
            __syncthreads();
            continue;
        }

        // Matching out of the words, completion, duals, cost.
        int *mb = fl0, *ma = fl1;
        for (int b = threadIdx.x; b < n; b += blockDim.x) mb[b] = -1;
        __syncthreads();
        for (int a = threadIdx.x; a < n; a += blockDim.x) {
            const unsigned long long w = pw[a];
            const int b = tag_of(w) > 0 ? row_of(w) : -1;
            ma[a] = b;
            if (b >= 0) mb[b] = a;
        }
        __syncthreads();
        // k-th free row (ascending) with the k-th free column (ascending)
        int *free_b = reinterpret_cast<int *>(ql0);
        int *free_a = free_b + n;
        int nfb = 0;
        for (int base = 0; base < n; base += blockDim.x) {
            const int b = base + threadIdx.x;
            const int f = (b < n && mb[b] < 0) ? 1 : 0;
            const int pos = block_scan_excl(f, s);
            if (f) free_b[nfb + pos] = b;
            nfb += s.total;
            __syncthreads();
        }
        int nfa = 0;
        for (int base = 0; base < n && nfa < nfb; base += blockDim.x) {
            const int a = base + threadIdx.x;
            const int f = (a < n && ma[a] < 0) ? 1 : 0;
            const int pos = block_scan_excl(f, s);
            if (f && nfa + pos < nfb) free_a[nfa + pos] = a;
            nfa += s.total;
            __syncthreads();
        }
        for (int k = threadIdx.x; k < nfb; k += blockDim.x) {
            mb[free_b[k]] = free_a[k];
            ma[free_a[k]] = free_b[k];
        }
        __syncthreads();
        double acc = 0.0;
        for (int b = threadIdx.x; b < n; b += blockDim.x) {
            p.row_to_col[D.v_off + b] = mb[b];
            p.y_row[D.v_off + b] = yb[b];
            double c;
            if (p.points) {
                c = dist_f64(p.XB + (long long)(D.v_off + b) * p.dim,
                             p.XA + (long long)(D.v_off + mb[b]) * p.dim, p.dim, p.squared);
            } else if (p.dt == PR_F64) {
                c = reinterpret_cast<const double *>(p.C)[D.c_off + (long long)b * n + mb[b]];
            } else {
                c = (double)reinterpret_cast<const float *>(p.C)[D.c_off + (long long)b * n + mb[b]];
            }
            acc = __dadd_rn(acc, c);
        }
        for (int a = threadIdx.x; a < n; a += blockDim.x) {
            p.col_to_row[D.v_off + a] = ma[a];
            p.y_col[D.v_off + a] = -(int)ks[a];
        }
        // fixed-order tree reduction of the per-thread partial sums
        double *part = reinterpret_cast<double *>(pw);
        __syncthreads();
        part[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + w]);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            p.costs[pi] = part[0];
            p.phases[pi] = phases;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long *)&p.ctl->phases, (unsigned long long)my_phases);
        atomicAdd((unsigned long long *)&p.ctl->rounds, (unsigned long long)my_rounds);
        atomicAdd(&p.ctl->bytes, s.bytes);
        atomicAdd(&p.ctl->rows, s.rows);
    }
}

size_t bsolve_smem(int n_max, int ldq_max, int threads) {
    // pw (8) + yb (4) + fl 2x(4) + ql 2x(8) + won (4) per row, keys 2 per column;
    // rows padded to a multiple of 8 as in k_bsolve; the cost reduction reuses
    // the front as one double per thread
    const size_t rows = (size_t)((n_max + 7) & ~7);
    const size_t state = rows * (8 + 4 + 8 + 16 + 4) + (size_t)ldq_max * 2;
    const size_t red = (size_t)threads * sizeof(double);
    return state > red ? state : red;
}

__global__ void k_binit(BCtl *ctl, unsigned *maxbits, int P) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        memset(ctl, 0, sizeof(BCtl));
        ctl->head.magic = kWsMagic;
    }
    for (int i = t; i < P; i += gridDim.x * blockDim.x) maxbits[i] = 0;
}

struct Plan {
    std::vector<BDesc> desc;
    std::vector<int> order;
    long long cb_elems = 0, c_elems = 0;
    int n_max = 0, ldq_max = 0, v_total = 0;
};

pr_status make_plan(int P, const int32_t *n_host, double eps, Plan &pl) {
    if (P < 1) return fail(PR_ERR_INVALID, "batched: n_problems must be >= 1");
    if (!n_host) return fail(PR_ERR_INVALID, "batched: NULL size array");
    pl.desc.resize(P);
    long long cb = 0, c = 0;
    long long v = 0;
    const long long K = eps > 0 ? (long long)floor(1.0 / eps) : 0;
    for (int i = 0; i < P; ++i) {
        const int n = n_host[i];
        if (n < 1 || n > kMaxN) return fail(PR_ERR_INVALID, "batched: problem %d has n = %d (need 1..%d)", i, n, kMaxN);
        BDesc &d = pl.desc[i];
        d.n = n;
        d.ldq = (n + 15) & ~15;  // rows start on 16 bytes in either storage type
        d.cb_off = cb;
        d.c_off = c;
        d.v_off = (int)v;
        d.T = (int)floor(eps * (double)n);
        d.cap = ((long long)n * (2 * K + 3)) / (d.T + 1) + 1;
        cb += (long long)n * d.ldq;
        c += (long long)n * n;
        v += n;
        pl.n_max = std::max(pl.n_max, n);
        pl.ldq_max = std::max(pl.ldq_max, d.ldq);
    }
    if (v > (1ll << 30)) return fail(PR_ERR_INVALID, "batched: too many rows in total");
    pl.cb_elems = cb;
    pl.c_elems = c;
    pl.v_total = (int)v;
    pl.order.resize(P);
    std::iota(pl.order.begin(), pl.order.end(), 0);
    // longest processing time first: larger problems start first
    std::stable_sort(pl.order.begin(), pl.order.end(),
                     [&](int a, int b) { return pl.desc[a].n > pl.desc[b].n; });
    return PR_OK;
}

struct Source {
    const void *C = nullptr;
    pr_dtype dt = PR_F64;
    const float *XA = nullptr, *XB = nullptr;
    int dim = 0;
    int squared = 1;
    bool points = false;
};

pr_status run_batched(const Source &src, int32_t P, const int32_t *n_host, double eps,
                      int32_t *row_to_col, int32_t *col_to_row, int32_t *y_row, int32_t *y_col,
                      double *costs, int64_t *phases, const pr_batched_tune *tune, pr_stats *stats,
                      void *ws, size_t ws_bytes, void *stream) {
    if (!row_to_col || !col_to_row || !y_row || !y_col || !costs || !phases)
        return fail(PR_ERR_INVALID, "batched: NULL output pointer");
    if (!(eps > 0.0 && eps < 1.0) || floor(1.0 / eps) > 32766.0)
        return fail(PR_ERR_INVALID, "batched: need 0 < eps < 1 and floor(1/eps) <= 32766");
    Plan pl;
    pr_status rc = make_plan(P, n_host, eps, pl);
    if (rc != PR_OK) return rc;
    const BLayout L = make_blayout(P, pl.cb_elems);
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < L.total)
        return fail(PR_ERR_WORKSPACE, "batched: workspace NULL, not 256-byte aligned or < %zu bytes", L.total);
    int threads = 256, per_sm_want = 0;
    if (tune) {
        if (tune->threads) threads = tune->threads;
        per_sm_want = tune->ctas_per_sm;
    }
    if (threads != 128 && threads != 256 && threads != 512 && threads != 1024)
        return fail(PR_ERR_INVALID, "batched: threads must be 128, 256, 512 or 1024");
    if (per_sm_want < 0) return fail(PR_ERR_INVALID, "batched: ctas_per_sm must be >= 0");

    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    BCtl *ctl = (BCtl *)(w + L.ctl);
    BDesc *d_desc = (BDesc *)(w + L.desc);
    int *d_order = (int *)(w + L.order);
    unsigned *d_max = (unsigned *)(w + L.maxbits);
    void *d_cb = w + L.cb;
    const bool cb8 = floor(1.0 / eps) <= (double)kMaxCbarByte;
    const DeviceInfo &di = device_info();

    k_binit<<<(P + 255) / 256, 256, 0, st>>>(ctl, d_max, P);
    PR_CUDA(cudaGetLastError());
    // problem table: copied from pageable host memory (waits for earlier work
    // on the stream; the host vectors may be freed on return)
    PR_CUDA(cudaMemcpyAsync(d_desc, pl.desc.data(), sizeof(BDesc) * P, cudaMemcpyHostToDevice, st));
    PR_CUDA(cudaMemcpyAsync(d_order, pl.order.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));

    const EpsSplit e = make_eps_split(eps);
    // a warp per row: 4 CTAs of 8 warps per SM (all resident at up to 64
    // registers a thread), fewer when there are fewer rows
    const int qgrid = std::max(1, std::min(di.sms * 4, (pl.v_total + 7) / 8));
    if (src.points) {
        // two and three dimensions have their own kernels (coordinates in
        // registers, several columns' loads in flight); any other runs the
        // column-at-a-time form
        const int D = src.dim == 2 ? 2 : src.dim == 3 ? 3 : 0;
        const void *kmax = D == 2 ? (const void *)k_bpoints_max<2> : D == 3 ? (const void *)k_bpoints_max<3>
                                                                              : (const void *)k_bpoints_max<0>;
        const void *kq = cb8 ? (D == 2 ? (const void *)k_bpoints_quant<2, uint8_t>
                                : D == 3 ? (const void *)k_bpoints_quant<3, uint8_t>
                                         : (const void *)k_bpoints_quant<0, uint8_t>)
                             : (D == 2 ? (const void *)k_bpoints_quant<2, uint16_t>
                                : D == 3 ? (const void *)k_bpoints_quant<3, uint16_t>
                                         : (const void *)k_bpoints_quant<0, uint16_t>);
        int dim_ = src.dim, sq_ = src.squared, P_ = P, rows_ = pl.v_total;
        const float *xa_ = src.XA, *xb_ = src.XB;
        const BDesc *dd_ = d_desc;
        unsigned *mx_ = d_max;
        void *amax[] = {(void *)&xa_, (void *)&xb_, (void *)&dim_, (void *)&sq_, (void *)&dd_, (void *)&P_,
                        (void *)&rows_, (void *)&mx_};
        PR_CUDA(cudaLaunchKernel(kmax, dim3(qgrid), dim3(256), amax, 0, st));
        const unsigned *cmx_ = d_max;
        void *cbp_ = d_cb;
        void *aq[] = {(void *)&xa_, (void *)&xb_, (void *)&dim_, (void *)&sq_, (void *)&dd_, (void *)&P_,
                      (void *)&rows_, (void *)&cmx_, (void *)&e, (void *)&cbp_};
        PR_CUDA(cudaLaunchKernel(kq, dim3(qgrid), dim3(256), aq, 0, st));
    } else if (src.dt == PR_F64) {
        if (cb8)
            k_bquant_matrix<double, uint8_t><<<qgrid, 256, 0, st>>>((const double *)src.C, d_desc, P, pl.v_total, e,
                                                                    (uint8_t *)d_cb, &ctl->head);
        else
            k_bquant_matrix<double, uint16_t><<<qgrid, 256, 0, st>>>((const double *)src.C, d_desc, P, pl.v_total,
                                                                     e, (uint16_t *)d_cb, &ctl->head);
    } else {
        if (cb8)
            k_bquant_matrix<float, uint8_t><<<qgrid, 256, 0, st>>>((const float *)src.C, d_desc, P, pl.v_total, e,
                                                                   (uint8_t *)d_cb, &ctl->head);
        else
            k_bquant_matrix<float, uint16_t><<<qgrid, 256, 0, st>>>((const float *)src.C, d_desc, P, pl.v_total, e,
                                                                    (uint16_t *)d_cb, &ctl->head);
    }
    PR_CUDA(cudaGetLastError());

    const size_t smem = bsolve_smem(pl.n_max, pl.ldq_max, threads);
    if (smem > (size_t)di.max_smem_optin)
        return fail(PR_ERR_INVALID, "batched: problem of n = %d does not fit shared memory", pl.n_max);
    // A warp scans a row in 2 KiB steps (a whole row of the largest size
    // for bytes; measured 9.5 % faster than 4 KiB steps on 512 problems of
    // 64..2048 points).
    const bool f7 = floor(1.0 / eps) <= 125.0;
    const void *kern = !cb8 ? (threads == 128   ? (const void *)k_bsolve<128, 4, uint16_t, false>
                               : threads == 256 ? (const void *)k_bsolve<256, 4, uint16_t, false>
                               : threads == 512 ? (const void *)k_bsolve<512, 4, uint16_t, false>
                                                : (const void *)k_bsolve<1024, 4, uint16_t, false>)
                       : f7 ? (threads == 128   ? (const void *)k_bsolve<128, 4, uint8_t, true>
                               : threads == 256 ? (const void *)k_bsolve<256, 4, uint8_t, true>
                               : threads == 512 ? (const void *)k_bsolve<512, 4, uint8_t, true>
                                                : (const void *)k_bsolve<1024, 4, uint8_t, true>)
                            : (threads == 128   ? (const void *)k_bsolve<128, 4, uint8_t, false>
                               : threads == 256 ? (const void *)k_bsolve<256, 4, uint8_t, false>
                               : threads == 512 ? (const void *)k_bsolve<512, 4, uint8_t, false>
                                                : (const void *)k_bsolve<1024, 4, uint8_t, false>);
    PR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return fail(PR_ERR_INVALID, "batched: solver CTA does not fit an SM");
    if (per_sm_want > 0 && per_sm_want < per_sm) per_sm = per_sm_want;
    int grid = di.sms * per_sm;
    if (grid > P) grid = P;

    BParams bp;
    bp.ctl = ctl;
    bp.desc = d_desc;
    bp.order = d_order;
    bp.maxbits = d_max;
    bp.cb = d_cb;
    bp.nprob = P;
    bp.n_max = pl.n_max;
    bp.ldq_max = pl.ldq_max;
    bp.C = src.C;
    bp.dt = src.dt;
    bp.XA = src.XA;
    bp.XB = src.XB;
    bp.dim = src.dim;
    bp.squared = src.squared;
    bp.points = src.points ? 1 : 0;
    bp.row_to_col = row_to_col;
    bp.col_to_row = col_to_row;
    bp.y_row = y_row;
    bp.y_col = y_col;
    bp.costs = costs;
    bp.phases = phases;
    cudaEvent_t ev0, ev1;
    kernel_events(&ev0, &ev1);
    if (ev0 && ev1) PR_CUDA(cudaEventRecord(ev0, st));
    {
        void *args[] = {(void *)&bp};
        PR_CUDA(cudaLaunchKernel(kern, dim3(grid), dim3(threads), args, smem, st));
    }
    if (ev0 && ev1) PR_CUDA(cudaEventRecord(ev1, st));

    if (stats) {
        BCtl h;
        PR_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(BCtl), cudaMemcpyDeviceToHost, st));
        PR_CUDA(cudaStreamSynchronize(st));
        stats->phases = h.phases;
        stats->rounds = h.rounds;
        stats->bytes_scanned = (int64_t)h.bytes;
        stats->rows_scanned = (int64_t)h.rows;
        stats->free_at_stop = 0;
        stats->threshold = 0;
        stats->loop_ctas = 0;
        stats->loop_cluster = 0;
        stats->cells_examined = 0;
        stats->barriers = 0;
        if (h.head.err != 0)
            return fail((pr_status)h.head.err, "batched: device reported %s", pr_status_string((pr_status)h.head.err));
    }
    return PR_OK;
}

}  // namespace
}  // namespace prot

using namespace prot;

extern "C" size_t pr_assign_batched_workspace(int32_t n_problems, const int32_t *n_host) {
    Plan pl;
    if (make_plan(n_problems, n_host, 0.5, pl) != PR_OK) return 0;
    return make_blayout(n_problems, pl.cb_elems).total;
}

extern "C" pr_status pr_assign_batched(const void *C, pr_dtype dt, int32_t n_problems,
                                       const int32_t *n_host, double eps, int32_t *row_to_col,
                                       int32_t *col_to_row, int32_t *y_row, int32_t *y_col,
                                       double *costs, int64_t *phases, const pr_batched_tune *tune,
                                       pr_stats *stats, void *ws, size_t ws_bytes, void *stream) {
    if (!C) return fail(PR_ERR_INVALID, "pr_assign_batched: NULL cost pointer");
    if (dt != PR_F32 && dt != PR_F64) return fail(PR_ERR_INVALID, "pr_assign_batched: bad dtype");
    Source src;
    src.C = C;
    src.dt = dt;
    return run_batched(src, n_problems, n_host, eps, row_to_col, col_to_row, y_row, y_col, costs,
                       phases, tune, stats, ws, ws_bytes, stream);
}

extern "C" pr_status pr_assign_batched_points(const float *XA, const float *XB, int32_t dim,
                                              pr_metric metric, int32_t n_problems,
                                              const int32_t *n_host, double eps,
                                              int32_t *row_to_col, int32_t *col_to_row,
                                              int32_t *y_row, int32_t *y_col, double *costs,
                                              int64_t *phases, const pr_batched_tune *tune,
                                              pr_stats *stats, void *ws, size_t ws_bytes,
                                              void *stream) {
    if (!XA || !XB) return fail(PR_ERR_INVALID, "pr_assign_batched_points: NULL point pointer");
    if (dim < 1 || dim > 4096) return fail(PR_ERR_INVALID, "pr_assign_batched_points: need 1 <= dim <= 4096");
    if (metric != PR_SQEUCLIDEAN && metric != PR_EUCLIDEAN)
        return fail(PR_ERR_INVALID, "pr_assign_batched_points: bad metric");
    Source src;
    src.XA = XA;
    src.XB = XB;
    src.dim = dim;
    src.squared = metric == PR_SQEUCLIDEAN ? 1 : 0;
    src.points = true;
    return run_batched(src, n_problems, n_host, eps, row_to_col, col_to_row, y_row, y_col, costs,
                       phases, tune, stats, ws, ws_bytes, stream);
}

// Launch-shape autotuner for the batched solver: runs the solve once with
// every candidate (threads per CTA x resident CTAs per SM) on the caller's
// batch, times each with CUDA events on `stream`, and returns the fastest.
// The outputs hold the last candidate's (identical) results.
extern "C" pr_status pr_assign_batched_autotune(const float *XA, const float *XB, int32_t dim,
                                                pr_metric metric, const void *C, pr_dtype dt,
                                                int32_t n_problems, const int32_t *n_host, double eps,
                                                int32_t *row_to_col, int32_t *col_to_row,
                                                int32_t *y_row, int32_t *y_col, double *costs,
                                                int64_t *phases, pr_batched_tune *best,
                                                float *best_ms, void *ws, size_t ws_bytes,
                                                void *stream) {
    if (!best || !best_ms) return fail(PR_ERR_INVALID, "pr_assign_batched_autotune: NULL result pointer");
    const bool points = XA && XB;
    if (!points && !C) return fail(PR_ERR_INVALID, "pr_assign_batched_autotune: give points or costs");
    cudaStream_t st = (cudaStream_t)stream;
    auto run = [&](const pr_batched_tune *t) -> pr_status {
        return points ? pr_assign_batched_points(XA, XB, dim, metric, n_problems, n_host, eps, row_to_col,
                                                 col_to_row, y_row, y_col, costs, phases, t, nullptr, ws,
                                                 ws_bytes, stream)
                      : pr_assign_batched(C, dt, n_problems, n_host, eps, row_to_col, col_to_row, y_row,
                                          y_col, costs, phases, t, nullptr, ws, ws_bytes, stream);
    };
    cudaEvent_t e0, e1;
    PR_CUDA(cudaEventCreate(&e0));
    PR_CUDA(cudaEventCreate(&e1));
    const int threads_c[] = {128, 256, 512, 1024};
    const int per_sm_c[] = {1, 2, 3, 4};
    float best_t = -1.0f;
    pr_batched_tune bt{0, 0};
    bool warmed = false;
    pr_status last_err = PR_OK;
    for (int th : threads_c) {
        for (int ps : per_sm_c) {
            pr_batched_tune t{th, ps};
            if (!warmed) {
                if (run(&t) != PR_OK) {
                    last_err = PR_ERR_INVALID;
                    continue;
                }
                warmed = true;
            }
            cudaEventRecord(e0, st);
            const pr_status rc = run(&t);
            cudaEventRecord(e1, st);
            if (rc != PR_OK) {  // this shape does not fit: skip it
                last_err = rc;
                cudaStreamSynchronize(st);
                continue;
            }
            PR_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            PR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (best_t < 0.0f || ms < best_t) {
                best_t = ms;
                bt = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_t < 0.0f) return fail(last_err != PR_OK ? last_err : PR_ERR_INVALID,
                                   "pr_assign_batched_autotune: no launch shape worked");
    // the solve with the chosen shape leaves its results in the outputs
    const pr_status rc = run(&bt);
    if (rc != PR_OK) return rc;
    *best = bt;
    *best_ms = best_t;
    return PR_OK;
}
