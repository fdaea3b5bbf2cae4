// rule_seq.cuh -- step (I) of Sec. 2.2 as the paper's sequential greedy
// (Sec. 3.2: the free rows in index order, each taking its first admissible
// column not yet in M'), computed by concurrent chains with no rounds.
// Included by assign.cu inside its namespace (it uses Params, Ctl and the
// proposal-word helpers there).
//
// Every column's proposal word (phase << 32 | ~row) is claimed by atomicMax,
// so within a phase a column is held by the lowest row that reached it.  A
// warp scans a row's columns in order against the phase's keys; at an
// admissible column it tries the word:
//   - a lower row holds it: the row scans on;
//   - a higher row holds it: that row is displaced, and the warp carries on
//     with the displaced row from the next column;
//   - the word is from an earlier phase: the column enters M' now, its key
//     rises (step III), and its partner in M, if any, is evicted (step II)
//     and queued for the next phase with its scan starting after the column.
// A row that reaches its end without a column is relabelled (step III) and
// queued for the next phase with its scan starting at column 0.
//
// Whatever order the chains run in, each column ends the phase held by the
// row the sequential greedy gives it.  By induction over the rows in index
// order: the columns held at the end by rows below b are those the greedy
// gives them, and every admissible column that b passed, or won and lost,
// is held at the end by a row below b (a column only ever passes to a lower
// row).  So one grid barrier per phase is the only synchronisation: none is
// needed between the proposals of one phase.
//
// Every CTA keeps the keys of the phase in shared memory.  A column that
// enters M' sets its bit in the bitmap of its phase (three bitmaps, by phase
// mod 3), and every CTA adds the previous phase's bits to its copy when a
// phase starts; the global keys, which columns raise during a phase, are
// read by no CTA until the loop ends.  Bitmap q % 3 is written in phase q,
// read at the start of phase q + 1 and cleared during phase q + 2, each
// step behind a grid barrier from the one before.
//
// The rows queued for the next phase go to a ring of 2 n_B entries of 16
// bytes (the list region; a relabelled row carries its new target) at
// positions from a counter that only grows: phase k's pushes fill
// [T_{k-1}, T_k), which phase k + 1 reads while its own pushes fill
// [T_k, T_{k+1}); each row is queued at most once per phase, so the two
// ranges never hold more than 2 n_B entries.

constexpr int kSeqUnroll = 4;  // 16-byte vectors per lane in flight per scan step
constexpr size_t kSeqMaxKeyBytes = 192 * 1024;  // shared memory for the phase's keys

// Admissible columns among the kPer columns [c, c + kPer) of one lane's
// vector: cbar + k == t, at or after the scan start s, below n_A.  Bytes take
// the packed byte test (exact per byte, a sum of 256 or more never matches);
// 16-bit values add lane-wise without carry between lanes (cbar + k <=
// 65534).
template <class CB>
__device__ __forceinline__ unsigned seq_marks(uint4 v, uint4 k, int t, int c, int s, int nA) {
    constexpr int kPer = 16 / (int)sizeof(CB);
    unsigned m;
    if (sizeof(CB) == 1)
        m = eq_mask8<false>(v, k, 0x01010101u * (uint32_t)t);
    else
        m = eq_mask(make_uint4(v.x + k.x, v.y + k.y, v.z + k.z, v.w + k.w), 0x00010001u * (uint32_t)t);
    const int lo = s > c ? s - c : 0, hi = nA - c < kPer ? nA - c : kPer;
    const unsigned range = (hi >= 32 ? ~0u : (1u << hi) - 1u) & ~((lo >= 32 ? ~0u : (1u << lo) - 1u));
    return lo >= hi ? 0u : (m & range);
}

// A row's scan runs on a group of wpr warps (1 to 16, a power of two): the
// fewer rows a phase has, the more warps each gets, so that the longest
// scan of the phase, which every phase waits for, is short.  The group
// finds its lowest candidate column through shared memory; groups of two or
// more warps synchronise on named barriers 1..8.
__device__ __forceinline__ void seq_group_sync(int gi, int wpr) {
    if (wpr == 1)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(1 + gi), "r"(wpr * 32) : "memory");
}

template <class CB>
__global__ void __launch_bounds__(kThreads, 1) k_seq(Params p) {
    extern __shared__ __align__(16) unsigned char seq_smem[];
    CB *ks = reinterpret_cast<CB *>(seq_smem);
    __shared__ unsigned long long s_push, s_sum;
    __shared__ int s_cand[2][kWarps];            // per warp: its lowest candidate, by parity
    __shared__ unsigned long long s_old[kWarps];  // per group: the word the leader's atomicMax returned
    constexpr int kPer = 16 / (int)sizeof(CB);   // columns per lane vector
    constexpr int kStep = 32 * kPer;             // columns per warp vector
    constexpr int kNone = 0x7FFFFFFF;
    constexpr int kNoTarget = -0x7FFFFFFF;  // an evicted row: its y(b) is in y_b
    Ctl *ctl = p.ctl;
    const unsigned G = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long total_warps = (long long)G * kWarps;
    const CB *cbm = static_cast<const CB *>(p.cb);
    int4 *ring = reinterpret_cast<int4 *>(p.lists);  // (row, scan start, target or kNoTarget, 0)
    const unsigned long long ring_n = 2ull * (unsigned long long)p.nB;
    unsigned gen = 0;
    long long phase = 0;
    unsigned long long nf = (unsigned long long)p.nB, start = 0, pushed = 0, sum = 0;
    unsigned long long cells = 0, bytes = 0;  // group leaders' counts
    for (int a = threadIdx.x; a < p.ldq; a += blockDim.x) ks[a] = 0;  // k(a) = 0 at the start

    auto push = [&](int row, int col, int tgt) {  // group leader only
        const unsigned long long pos = atomicAdd(&ctl->seq_tail, 1ull);
        ring[pos % ring_n] = make_int4(row, col, tgt, 0);
        atomicAdd(&s_push, 1ull);
    };

    for (;;) {
        if ((long long)nf <= p.T) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->free_at_stop = (int)nf;
            break;
        }
        if (phase >= p.phase_cap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                ctl->free_at_stop = (int)nf;
                record_error(&ctl->head, PR_ERR_NO_CONVERGENCE);
            }
            break;
        }
        ++phase;
        const unsigned ph = (unsigned)phase;
        const int W = p.won_words;
        const unsigned long long t0 = p.profile ? ptimer() : 0;
        // warps per row: the largest power of two <= total warps / rows, in [1, 16]
        int wpr = 1;
        while (wpr < kWarps && (unsigned long long)(2 * wpr) * nf <= (unsigned long long)total_warps) wpr *= 2;
        const int gi = warp / wpr, wi = warp % wpr;  // group in the CTA, warp in the group
        const bool leader = wi == 0 && lane == 0;
        const long long groups = total_warps / wpr;
        const long long rank = (long long)gi * G + blockIdx.x;  // CTA-minor: rows spread over the CTAs
        const int gstep = kSeqUnroll * wpr * kStep;           // columns per group scan step
        // the group's first row, loaded before the key update below
        int4 e = make_int4((int)rank, 0, 0, 0);  // phase 1: every row, y(b) = 1, from column 0
        if (phase > 1 && (unsigned long long)rank < nf) e = ring[(start + rank) % ring_n];
        if (phase > 1) {  // the columns that entered M' in the previous phase: k(a) += 1
            const unsigned *prev = p.won + (size_t)((ph - 1) % 3) * W;
            for (int w = threadIdx.x; w < W; w += blockDim.x) {
                unsigned bits = prev[w];
                while (bits) {
                    const int j = __ffs(bits) - 1;
                    bits &= bits - 1;
                    ks[w * 32 + j] = (CB)(ks[w * 32 + j] + 1);
                }
            }
            unsigned *old = p.won + (size_t)((ph + 1) % 3) * W;  // written two phases ago
            for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < W;
                 w += (long long)G * blockDim.x)
                old[w] = 0;
        }
        unsigned *won = p.won + (size_t)(ph % 3) * W;
        if (threadIdx.x == 0) s_push = 0;
        __syncthreads();
        const unsigned long long t1 = p.profile ? ptimer() : 0;

        int par = 0;
        for (unsigned long long i = (unsigned long long)rank; i < nf; i += (unsigned long long)groups) {
            int b = e.x, s = e.y, t = e.z;
            if (t == kNoTarget) t = p.y_b[b] - 1;
            const unsigned long long nx = i + (unsigned long long)groups;  // the group's next row
            if (nx < nf) e = phase > 1 ? ring[(start + nx) % ring_n] : make_int4((int)nx, 0, 0, 0);
            for (;;) {  // one chain: row b from column s, then any row it displaces
                const CB *row = cbm + (size_t)b * p.ldq;
                int found = -1, other = -1;
                bool first = false;
                for (int base = (s / gstep) * gstep; base < p.nA && found < 0; base += gstep) {
                    uint4 v[kSeqUnroll];
                    unsigned m[kSeqUnroll];
#pragma unroll
                    for (int u = 0; u < kSeqUnroll; ++u) {
                        const int c = base + ((u * wpr + wi) * 32 + lane) * kPer;
                        v[u] = c < p.nA ? *reinterpret_cast<const uint4 *>(row + c) : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int u = 0; u < kSeqUnroll; ++u) {
                        const int c = base + ((u * wpr + wi) * 32 + lane) * kPer;
                        m[u] = c < p.nA
                                   ? seq_marks<CB>(v[u], *reinterpret_cast<const uint4 *>(ks + c), t, c, s, p.nA)
                                   : 0u;
                    }
                    if (leader) bytes += (unsigned long long)kSeqUnroll * wpr * 512;
                    // the candidates of this step, lowest first
                    for (;;) {
                        int mine = kNone;
#pragma unroll
                        for (int u = kSeqUnroll - 1; u >= 0; --u)
                            if (m[u]) mine = base + ((u * wpr + wi) * 32 + lane) * kPer + __ffs(m[u]) - 1;
                        const int wmin = __reduce_min_sync(0xFFFFFFFFu, mine);
                        int a = wmin;
                        if (wpr > 1) {
                            if (lane == 0) s_cand[par][warp] = wmin;
                            seq_group_sync(gi, wpr);
                            for (int k = 0; k < wpr; ++k) a = min(a, s_cand[par][gi * wpr + k]);
                            par ^= 1;
                        }
                        if (a == kNone) break;  // none in this step
                        unsigned long long old = 0;
                        if (leader) old = atomicMax(p.prop + a, word_of(ph, b));
                        if (wpr > 1) {
                            if (leader) s_old[gi] = old;
                            seq_group_sync(gi, wpr);
                            old = s_old[gi];
                        } else {
                            old = __shfl_sync(0xFFFFFFFFu, old, 0);
                        }
                        if (tag_of(old) == ph && row_of(old) < b) {  // a lower row holds a
                            if (mine == a) {
#pragma unroll
                                for (int u = 0; u < kSeqUnroll; ++u)
                                    if (m[u]) {
                                        m[u] &= m[u] - 1;
                                        break;
                                    }
                            }
                            continue;
                        }
                        found = a;
                        first = tag_of(old) != ph;
                        other = tag_of(old) > 0 ? row_of(old) : -1;
                        break;
                    }
                }
                if (leader) cells += (unsigned long long)((found >= 0 ? found + 1 : p.nA) - s);
                if (found < 0) {  // no admissible column left: y(b) += eps, next phase from column 0
                    if (leader) {
                        p.y_b[b] = t + 2;
                        push(b, 0, t + 1);
                    }
                    break;
                }
                if (first) {  // found enters M' now; its partner in M leaves M
                    if (leader) {
                        p.ka[found] = (uint16_t)(p.ka[found] + 1);
                        atomicOr(won + (found >> 5), 1u << (found & 31));
                        if (other >= 0) push(other, found + 1, kNoTarget);
                    }
                    break;
                }
                b = other;  // displaced: its columns before found are settled
                s = found + 1;
                t = p.y_b[b] - 1;
            }
        }
        __syncthreads();
        const unsigned long long mine = s_push;
        unsigned long long t2 = 0;
        if (p.profile && threadIdx.x == 0) {
            // PR_PROFILE=1: per phase the maximum over CTAs of the key update,
            // the chains and both, in rotating slots of prof_slot (phase % 3)
            t2 = ptimer();
            unsigned long long *slot = &ctl->prof_slot[0][0] + (ph % 3) * 4;
            atomicMax(slot + 0, t1 - t0);
            atomicMax(slot + 1, t2 - t1);
            atomicMax(slot + 2, t2 - t0);
        }
        if (!grid_sum_barrier(&ctl->bar_slot[0][0], &ctl->head, gen, G, p.spin_limit, mine, sum)) break;
        if (p.profile && threadIdx.x == 0) {
            const unsigned long long t3 = ptimer();
            if (blockIdx.x == 0) {
                unsigned long long *slot = &ctl->prof_slot[0][0] + (ph % 3) * 4;
                // the slot read at the previous barrier is written next in phase ph + 2
                unsigned long long *next = &ctl->prof_slot[0][0] + ((ph + 2) % 3) * 4;
                for (int k = 0; k < 3; ++k) {
                    ctl->prof_max[k] += slot[k];
                    next[k] = 0;
                }
                ctl->prof_own[0] += t1 - t0;
                ctl->prof_own[1] += t2 - t1;
                ctl->prof_own[2] += t3 - t2;
                ctl->prof_own[3] += wpr;
                ctl->prof_rounds += 1;
            }
        }
        start = pushed;
        pushed += sum;
        nf = sum;
    }
    // counters: every group leader holds its group's counts
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    if (cells) atomicAdd(&s_sum, cells);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(&ctl->cells, s_sum);
    __syncthreads();
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    if (bytes) atomicAdd(&s_sum, bytes);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(&ctl->bytes, s_sum);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->phases = phase;
        ctl->rounds = phase;  // one pass of step I per phase
        ctl->barriers = gen;
    }
}
