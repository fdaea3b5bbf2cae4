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
// step behind a grid barrier from the one before.  The rows queued for the next
// phase go to a ring of 2 n_B entries (the pool region) at positions from a
// counter that only grows: phase k's pushes fill [T_{k-1}, T_k), which
// phase k + 1 reads while phase k + 1's own pushes fill [T_k, T_{k+1});
// each row is queued at most once per phase, so the two ranges never hold
// more than 2 n_B entries.

constexpr int kSeqUnroll = 4;  // 16-byte vectors per lane in flight per scan step
constexpr size_t kSeqMaxKeyBytes = 192 * 1024;  // shared memory for the phase's keys

// Admissible columns among the kPer columns [c, c + kPer) of one lane's
// vector: cbar + k == t, at or after the scan start s, below n_A.
template <class CB>
__device__ __forceinline__ unsigned seq_marks(uint4 v, uint4 k, int t, int c, int s, int nA) {
    constexpr int kPer = 16 / (int)sizeof(CB);
    const uint32_t vq[4] = {v.x, v.y, v.z, v.w};
    const uint32_t kq[4] = {k.x, k.y, k.z, k.w};
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        int cv, kv;
        if (sizeof(CB) == 1) {
            cv = (int)((vq[j >> 2] >> (8 * (j & 3))) & 0xFFu);
            kv = (int)((kq[j >> 2] >> (8 * (j & 3))) & 0xFFu);
        } else {
            cv = (int)((vq[j >> 1] >> (16 * (j & 1))) & 0xFFFFu);
            kv = (int)((kq[j >> 1] >> (16 * (j & 1))) & 0xFFFFu);
        }
        const int col = c + j;
        if (col >= s && col < nA && cv + kv == t) m |= 1u << j;
    }
    return m;
}

template <class CB>
__global__ void __launch_bounds__(kThreads, 1) k_seq(Params p) {
    extern __shared__ __align__(16) unsigned char seq_smem[];
    CB *ks = reinterpret_cast<CB *>(seq_smem);
    __shared__ unsigned long long s_push, s_sum;
    constexpr int kPer = 16 / (int)sizeof(CB);  // columns per lane vector
    constexpr int kStep = 32 * kPer;            // columns per warp vector
    Ctl *ctl = p.ctl;
    const unsigned G = gridDim.x;
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)G * (blockDim.x >> 5);
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const CB *cbm = static_cast<const CB *>(p.cb);
    int2 *ring = p.pool;
    const unsigned long long ring_n = 2ull * (unsigned long long)p.nB;
    unsigned gen = 0;
    long long phase = 0;
    unsigned long long nf = (unsigned long long)p.nB, start = 0, pushed = 0, sum = 0;
    unsigned long long cells = 0, bytes = 0;  // lane 0's counts
    bool ok = true;
    for (int a = threadIdx.x; a < p.ldq; a += blockDim.x) ks[a] = 0;  // k(a) = 0 at the start

    auto push = [&](int row, int col) {  // lane 0 only
        const unsigned long long pos = atomicAdd(&ctl->seq_tail, 1ull);
        ring[pos % ring_n] = make_int2(row, col);
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

        for (unsigned long long i = (unsigned long long)gw; i < nf; i += (unsigned long long)nw) {
            int b, s;
            if (phase == 1) {
                b = (int)i;
                s = 0;
            } else {
                const int2 e = ring[(start + i) % ring_n];
                b = e.x;
                s = e.y;
            }
            int t = p.y_b[b] - 1;
            for (;;) {  // one chain: row b from column s, then any row it displaces
                const CB *row = cbm + (size_t)b * p.ldq;
                int found = -1, other = -1;
                bool first = false;
                for (int base = (s / kStep) * kStep; base < p.nA && found < 0; base += kSeqUnroll * kStep) {
                    uint4 v[kSeqUnroll];
#pragma unroll
                    for (int u = 0; u < kSeqUnroll; ++u) {
                        const int c = base + u * kStep + lane * kPer;
                        v[u] = c < p.nA ? *reinterpret_cast<const uint4 *>(row + c) : make_uint4(0, 0, 0, 0);
                    }
                    if (lane == 0) bytes += (unsigned long long)kSeqUnroll * 512;
#pragma unroll
                    for (int u = 0; u < kSeqUnroll; ++u) {
                        if (found >= 0) break;
                        const int c = base + u * kStep + lane * kPer;
                        unsigned m = 0;
                        if (c < p.nA)
                            m = seq_marks<CB>(v[u], *reinterpret_cast<const uint4 *>(ks + c), t, c, s, p.nA);
                        // the candidates of this vector step, in column order
                        for (;;) {
                            const unsigned bal = __ballot_sync(0xFFFFFFFFu, m != 0);
                            if (!bal) break;
                            const int src = __ffs(bal) - 1;
                            const unsigned ms = __shfl_sync(0xFFFFFFFFu, m, src);
                            const int a = base + u * kStep + src * kPer + (__ffs(ms) - 1);
                            unsigned long long old = 0;
                            if (lane == 0) old = atomicMax(p.prop + a, word_of(ph, b));
                            old = __shfl_sync(0xFFFFFFFFu, old, 0);
                            if (tag_of(old) == ph && row_of(old) < b) {  // a lower row holds a
                                if (lane == src) m &= m - 1;
                                continue;
                            }
                            found = a;
                            first = tag_of(old) != ph;
                            other = tag_of(old) > 0 ? row_of(old) : -1;
                            break;
                        }
                    }
                }
                if (lane == 0) cells += (unsigned long long)((found >= 0 ? found + 1 : p.nA) - s);
                if (found < 0) {  // no admissible column left: y(b) += eps, next phase from column 0
                    if (lane == 0) {
                        p.y_b[b] = t + 2;
                        push(b, 0);
                    }
                    break;
                }
                if (first) {  // found enters M' now; its partner in M leaves M
                    if (lane == 0) {
                        p.ka[found] = (uint16_t)(p.ka[found] + 1);
                        atomicOr(won + (found >> 5), 1u << (found & 31));
                        if (other >= 0) push(other, found + 1);
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
        if (!grid_sum_barrier(&ctl->bar_slot[0][0], &ctl->head, gen, G, p.spin_limit, mine, sum)) {
            ok = false;
            break;
        }
        start = pushed;
        pushed += sum;
        nf = sum;
    }
    (void)ok;
    // counters: lane 0 of every warp holds its warp's counts
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    if (lane == 0 && cells) atomicAdd(&s_sum, cells);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(&ctl->cells, s_sum);
    __syncthreads();
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    if (lane == 0 && bytes) atomicAdd(&s_sum, bytes);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(&ctl->bytes, s_sum);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->phases = phase;
        ctl->rounds = phase;  // one pass of step I per phase
        ctl->barriers = gen;
    }
}
