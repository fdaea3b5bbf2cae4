// rule_ii.cuh -- step (I) of Sec. 2.2 by Israeli and Itai's randomized
// maximal matching (A. Israeli, A. Itai, "A fast and simple randomized
// parallel algorithm for maximal matching", IPL 22, 1986), which Sec. 3.2
// names for the O(log n) parallel bound of a phase.  Included by assign.cu
// inside its namespace (it uses Params, Ctl and the launch plumbing there).
//
// One iteration on the admissible graph of the phase's live free rows and
// the columns not yet in M' (an edge (b, a): y(a) + y(b) = cbar + 1):
//   1. every vertex with an edge points to one neighbour, chosen uniformly;
//   2. every vertex pointed at keeps one of the pointers, chosen uniformly;
//   3. every vertex is left with at most two edges (the one it points along
//      if kept, the one it kept); it picks one, uniformly, and an edge picked
//      at both ends joins M'.
// Matched rows and rows without an edge leave; iterations go on while some
// row has an edge, so M' ends maximal.  Step II/III then run as for the
// other rules.
//
// A uniform choice is the candidate of least key, key = (draw >> 24) << 24 |
// candidate index (40 random bits, then the index, which also settles
// ties); a choice between two edges takes the low bit of a draw.  A draw is
// three SplitMix64 rounds (Steele, Lea and Flood 2014) over (step, phase,
// iteration), then the vertex id, then the other end's index; vertex ids
// are b for row b and 2^24 + a for column a.  With keys, steps 1 and 2 are
// atomicMin on 64-bit words, and the whole rule is deterministic: the
// oracle's OR_MODE_ISRAELI_ITAI gives the same M' in every phase.
//
// Layout: one cooperative grid (one CTA per SM); a warp scans a live row
// (each lane 8 columns per step), threads sweep rows and columns for steps
// 2 and 3; every step ends at a grid barrier.  The matching M is kept in two
// int arrays and handed to k_decode as proposal words at the end.

constexpr int kIIMaxIters = 4096;  // iterations per phase before PR_ERR_NO_CONVERGENCE
constexpr unsigned kIICol = 1u << 24;
constexpr unsigned long long kIINone = ~0ull;

__device__ __forceinline__ unsigned long long ii_splitmix(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__device__ __forceinline__ unsigned long long ii_draw(unsigned step, unsigned phase, unsigned it, unsigned u, unsigned v) {
    unsigned long long x = ii_splitmix(((unsigned long long)step << 56) ^ ((unsigned long long)phase << 28) ^ it);
    x = ii_splitmix(x ^ u);
    return ii_splitmix(x ^ v);
}
__device__ __forceinline__ unsigned long long ii_key(unsigned step, unsigned phase, unsigned it, unsigned u, unsigned v) {
    return ((ii_draw(step, phase, it, u, v) >> 24) << 24) | (unsigned long long)(v & 0xFFFFFFu);
}

// Per-iteration and per-phase state, carved from the workspace's list region.
struct IIWork {
    unsigned long long *cp;   // [nA] step 1: a column's pointer, as the key of its row
    unsigned long long *cin;  // [nA] step 2: the pointer a column keeps (key of the row)
    unsigned long long *rin;  // [nB] step 2: the pointer a row keeps (key of the column)
    int *mB, *mA;             // the matching M (-1: free)
    int *act;                 // [nB] live in this phase's step I
    int *mate;                // [nB] partner in M' (-1: none)
    int *taken;               // [nA] in M'
    int *rp;                  // [nB] step 1: the column a row points to (-1: no edge)
    int *rc, *cc;             // step 3 picks; rc = -2 marks a row evicted at the phase end
};

__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, unsigned long long *sh) {
    __syncthreads();
    if (threadIdx.x == 0) *sh = 0;
    __syncthreads();
    if (v) atomicAdd(sh, v);
    __syncthreads();
    return *sh;
}

template <class CB>
__global__ void __launch_bounds__(kThreads, 1) k_ii(Params p, IIWork w) {
    __shared__ unsigned long long bsum;
    Ctl *ctl = p.ctl;
    const unsigned G = gridDim.x;
    const long long nth = (long long)G * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const long long gw = t0 >> 5, nw = nth >> 5;
    const CB *cbm = static_cast<const CB *>(p.cb);
    unsigned gen = 0;
    long long phase = 0, rounds = 0;
    unsigned long long cells = 0, sum = 0;
    bool ok = true;
    for (long long b = t0; b < p.nB; b += nth) {
        w.mB[b] = -1;
        w.rin[b] = kIINone;
    }
    for (long long a = t0; a < p.nA; a += nth) {
        w.mA[a] = -1;
        w.cp[a] = kIINone;
        w.cin[a] = kIINone;
    }
    for (;;) {
        // ---- phase start: B' = the free rows ----
        unsigned long long nf = 0;
        for (long long b = t0; b < p.nB; b += nth) {
            const int f = w.mB[b] < 0 ? 1 : 0;
            w.act[b] = f;
            w.mate[b] = -1;
            nf += f;
        }
        for (long long a = t0; a < p.nA; a += nth) w.taken[a] = 0;
        const unsigned long long nfb = block_sum(nf, &bsum);
        if (!grid_sum_barrier(&ctl->bar_slot[0][0], &ctl->head, gen, G, p.spin_limit, nfb, sum)) {
            ok = false;
            break;
        }
        if ((long long)sum <= p.T) {
            if (t0 == 0) ctl->free_at_stop = (int)sum;
            break;
        }
        if (phase >= p.phase_cap) {
            if (t0 == 0) {
                ctl->free_at_stop = (int)sum;
                record_error(&ctl->head, PR_ERR_NO_CONVERGENCE);
            }
            break;
        }
        ++phase;
        const unsigned ph = (unsigned)phase;
        for (unsigned it = 1;; ++it) {
            if (it > (unsigned)kIIMaxIters) {
                if (t0 == 0) record_error(&ctl->head, PR_ERR_NO_CONVERGENCE);
                ok = false;
                break;
            }
            // step 1: a warp per live row; every edge to a column not in M'
            unsigned long long live = 0;
            for (long long b = gw; b < p.nB; b += nw) {
                if (!w.act[b]) continue;
                const int t = p.y_b[b] - 1;
                const CB *row = cbm + (size_t)b * p.ldq;
                unsigned long long best = kIINone;
                for (int c0 = lane * 8; c0 < p.nA; c0 += 256) {
                    uint32_t cv[8], kv[8];
                    if (sizeof(CB) == 1) {
                        const uint2 x = *reinterpret_cast<const uint2 *>(row + c0);
                        for (int j = 0; j < 8; ++j) cv[j] = ((j < 4 ? x.x : x.y) >> (8 * (j & 3))) & 0xFFu;
                    } else {
                        const uint4 x = *reinterpret_cast<const uint4 *>(row + c0);
                        const uint32_t q[4] = {x.x, x.y, x.z, x.w};
                        for (int j = 0; j < 8; ++j) cv[j] = (q[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
                    }
                    const uint4 k4 = *reinterpret_cast<const uint4 *>(p.ka + c0);
                    const uint32_t kq[4] = {k4.x, k4.y, k4.z, k4.w};
                    for (int j = 0; j < 8; ++j) kv[j] = (kq[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
                    for (int j = 0; j < 8; ++j) {
                        const int a = c0 + j;
                        if (a >= p.nA || (int)(cv[j] + kv[j]) != t || w.taken[a]) continue;
                        const unsigned long long kr = ii_key(1, ph, it, (unsigned)b, (unsigned)a);
                        best = kr < best ? kr : best;
                        atomicMin(w.cp + a, ii_key(1, ph, it, kIICol + (unsigned)a, (unsigned)b));
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, best, o);
                    best = y < best ? y : best;
                }
                if (lane == 0) {
                    cells += (unsigned long long)p.nA;
                    if (best == kIINone) {
                        w.rp[b] = -1;
                        w.act[b] = 0;  // no edge left: relabelled at the phase end
                    } else {
                        w.rp[b] = (int)(best & 0xFFFFFFu);
                        ++live;
                    }
                }
            }
            const unsigned long long lb = block_sum(live, &bsum);
            if (!grid_sum_barrier(&ctl->bar_slot[0][0], &ctl->head, gen, G, p.spin_limit, lb, sum)) {
                ok = false;
                break;
            }
            if (sum == 0) break;  // no row has an edge: M' is maximal
            ++rounds;
            // step 2: every vertex pointed at keeps the pointer of least key
            for (long long b = t0; b < p.nB; b += nth)
                if (w.act[b]) {
                    const int a = w.rp[b];
                    atomicMin(w.cin + a, ii_key(2, ph, it, kIICol + (unsigned)a, (unsigned)b));
                }
            for (long long a = t0; a < p.nA; a += nth) {
                const unsigned long long k = w.cp[a];
                if (k != kIINone) {
                    const unsigned b = (unsigned)(k & 0xFFFFFFu);
                    atomicMin(w.rin + b, ii_key(2, ph, it, b, (unsigned)a));
                }
            }
            if (!grid_sum_barrier(&ctl->bar_slot[0][0], &ctl->head, gen, G, p.spin_limit, 0, sum)) {
                ok = false;
                break;
            }
            // step 3: every vertex picks one of its kept edges
            for (long long b = t0; b < p.nB; b += nth) {
                int pick = -1;
                if (w.act[b]) {
                    const int a = w.rp[b];
                    const unsigned long long ci = w.cin[a];
                    const int out = (ci != kIINone && (long long)(ci & 0xFFFFFFu) == b) ? a : -1;
                    const unsigned long long ri = w.rin[b];
                    const int in = ri != kIINone ? (int)(ri & 0xFFFFFFu) : -1;
                    if (out >= 0 && in >= 0)
                        pick = (ii_draw(3, ph, it, (unsigned)b, 0) & 1ull) ? in : out;
                    else
                        pick = out >= 0 ? out : in;
                }
                w.rc[b] = pick;
            }
            for (long long a = t0; a < p.nA; a += nth) {
                int pick = -1;
                if (!w.taken[a]) {
                    int out = -1;
                    const unsigned long long k = w.cp[a];
                    if (k != kIINone) {
                        const int b = (int)(k & 0xFFFFFFu);
                        const unsigned long long ri = w.rin[b];
                        if (ri != kIINone && (long long)(ri & 0xFFFFFFu) == a) out = b;
                    }
                    const unsigned long long ci = w.cin[a];
                    const int in = ci != kIINone ? (int)(ci & 0xFFFFFFu) : -1;
                    if (out >= 0 && in >= 0)
                        pick = (ii_draw(3, ph, it, kIICol + (unsigned)a, 0) & 1ull) ? in : out;
                    else
                        pick = out >= 0 ? out : in;
                }
                w.cc[a] = pick;
            }
            if (!grid_sum_barrier(&ctl->bar_slot[0][0], &ctl->head, gen, G, p.spin_limit, 0, sum)) {
                ok = false;
                break;
            }
            // an edge picked at both ends joins M'; the iteration's words are
            // cleared for the next one
            for (long long b = t0; b < p.nB; b += nth) {
                const int a = w.rc[b];
                if (a >= 0 && w.cc[a] == (int)b) {
                    w.mate[b] = a;
                    w.taken[a] = 1;
                    w.act[b] = 0;
                }
                w.rin[b] = kIINone;
            }
            for (long long a = t0; a < p.nA; a += nth) {
                w.cp[a] = kIINone;
                w.cin[a] = kIINone;
            }
            if (!grid_sum_barrier(&ctl->bar_slot[0][0], &ctl->head, gen, G, p.spin_limit, 0, sum)) {
                ok = false;
                break;
            }
        }
        if (!ok) break;
        // step II (add M', the old partners of its columns become free) and
        // step III (y(a) -= eps on M', y(b) += eps for the rest of B'): first
        // mark the evicted rows, then apply
        for (long long b = t0; b < p.nB; b += nth) {
            const int a = w.mate[b];
            if (a >= 0) {
                const int old = w.mA[a];
                if (old >= 0) w.rc[old] = -2;
            } else if (w.mB[b] < 0) {
                p.y_b[b] += 1;
            }
        }
        if (!grid_sum_barrier(&ctl->bar_slot[0][0], &ctl->head, gen, G, p.spin_limit, 0, sum)) {
            ok = false;
            break;
        }
        for (long long b = t0; b < p.nB; b += nth) {
            const int a = w.mate[b];
            if (a >= 0) {
                w.mA[a] = (int)b;
                w.mB[b] = a;
                p.ka[a] = (uint16_t)(p.ka[a] + 1);
            } else if (w.rc[b] == -2) {
                w.mB[b] = -1;
            }
            w.rc[b] = -1;
        }
        if (!grid_sum_barrier(&ctl->bar_slot[0][0], &ctl->head, gen, G, p.spin_limit, 0, sum)) {
            ok = false;
            break;
        }
    }
    // the matching as k_decode's proposal words
    if (ok)
        for (long long a = t0; a < p.nA; a += nth)
            p.prop[a] = w.mA[a] >= 0 ? word_of(1, w.mA[a]) : word_of(0, -1);
    const unsigned long long cb = block_sum(cells, &bsum);
    if (threadIdx.x == 0 && cb) {
        atomicAdd(&ctl->cells, cb);
        atomicAdd(&ctl->bytes, cb * sizeof(CB));  // every live row is read whole each round
    }
    if (t0 == 0) {
        ctl->phases = phase;
        ctl->rounds = rounds;
        ctl->barriers = gen;
    }
}
