// S5 track following: Kalman-filter following of each seed across the pad rows, one thread per
// track candidate (arxiv 1712.09434 section 3).  Every accept/reject decision is taken by an
// integer steady-state Kalman filter (alpha-beta-gamma = 1/2, 1/8, 1/32 on a Q16 state, floor
// shifts, int64) so that the hit lists are bit-identical to an independent FP64 implementation;
// the floating-point Kalman filter is used for the parameters only (S8).
//
// The filter runs along the whole chain, then extends it row by row outwards, then (re-initialised
// from the other end) inwards: predict, look up the nearest cluster (minimum (d^2, index)) within a
// radius that grows with consecutive misses in the row's Z-slab grid, update.  A candidate is
// stored as one cluster per row (-1 for a miss) between its first and last row.  The chains are
// taken in an order that groups chains of equal length and nearby start rows in a warp (below).
#include "tpc_common.cuh"

namespace tpc {

namespace {

struct Abg {
    long long p, v, a;
};

// state at m0 with the velocity of the step to m1, drow = 1 or 2 rows further (2 across a row that
// a link skips; the division is exact)
__device__ __forceinline__ void abg_init(Abg &f, long long m0, long long m1, int drow) {
    f.p = m0 * 65536;
    f.v = (m1 - m0) * (65536 / drow);
    f.a = 0;
}
__device__ __forceinline__ void abg_predict(Abg &f) {
    f.p += f.v + (f.a >> 1);
    f.v += f.a;
}
__device__ __forceinline__ void abg_update(Abg &f, long long m) {
    const long long e = m * 65536 - f.p;
    f.p += e >> 1;
    f.v += e >> 3;
    f.a += e >> 5;
}
__device__ __forceinline__ int q16_round(long long p) { return (int)((p + 32768) >> 16); }
__device__ __forceinline__ int slab_of(int z) { int s = z >> ZB_SHIFT; return s < NZB - 1 ? s : NZB - 1; }

__device__ __forceinline__ int lower_y(const int32_t *yz, int lo, int hi, int y) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)(int16_t)(__ldg(yz + mid) & 0xffff) < y) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Nearest cluster of a row bin to (py, pz) with d^2 <= w^2: row-local index, or -1; its packed
// (Y, Z) goes to *yz (the grid payload, so the cluster arrays need not be read again).
__device__ int nearest(const Work &W, int bin, int py, int pz, int w, int32_t *yz_out) {
    const int c0 = __ldg(W.bin_off + bin);
    const int32_t *yz = W.gyz + pstart_of(c0, bin);
    const uint16_t *loc = W.gloc + pstart_of(c0, bin);
    const uint16_t *zo = W.zoff + (size_t)bin * ZOFF_STRIDE;
    const int zl = slab_of(max(pz - w, 0)), zh = slab_of(pz + w);
    const long long w2 = (long long)w * w;
    long long bd = w2 + 1;
    int bl = 0x7fffffff;
    int32_t bv = 0;
    for (int s = zl; s <= zh; s++) {
        const int hi = __ldg(zo + s + 1);
        for (int i = lower_y(yz, __ldg(zo + s), hi, py - w); i < hi; i++) {
            const int32_t v = __ldg(yz + i);
            const int y = (int16_t)(v & 0xffff);
            if (y > py + w) break;
            const long long dy = y - py, dz = (int)((uint32_t)v >> 16) - pz;
            const long long d2 = dy * dy + dz * dz;
            if (d2 > w2) continue;
            const int l = __ldg(loc + i);
            if (d2 < bd || (d2 == bd && l < bl)) { bd = d2; bl = l; bv = v; }
        }
    }
    *yz_out = bv;
    return bl == 0x7fffffff ? -1 : bl;
}

// Extend from the filter state (already at row `row_last`) in direction dir; writes slots.
// Returns the number of clusters found and the row of the last one in *row_end.
__device__ int extend(const Work &W, const DevGeom &g, Abg &fy, Abg &fz, int rowbase_bin, int row_last, int dir,
                      int32_t *slots, int *row_end) {
    int n = 0, misses = 0;
    *row_end = row_last;
    for (int row = row_last + dir; row >= 0 && row < g.n_rows; row += dir) {
        abg_predict(fy);
        abg_predict(fz);
        const int py = q16_round(fy.p), pz = q16_round(fz.p);
        const long long av = fy.v < 0 ? -fy.v : fy.v;
        if (abs(py) > g.ymax[row] || pz < 0 || pz > g.zmax || av > (long long)V_MAX * 65536) break;
        const int w = W_F0 + W_F1 * misses;
        int32_t v;
        const int l = nearest(W, rowbase_bin + row, py, pz, w, &v);
        if (l >= 0) {
            const int h = __ldg(W.bin_off + rowbase_bin + row) + l;
            abg_update(fy, (int16_t)(v & 0xffff));
            abg_update(fz, (int)((uint32_t)v >> 16));
            slots[row] = h;
            *row_end = row;
            n++;
            misses = 0;
        } else {
            slots[row] = -1;
            if (++misses >= M_MISS) break;
        }
    }
    return n;
}

// Order in which the following takes the chains: per (event, sector), by groups of 16 start rows
// and inside a group by decreasing chain length (lengths of 127 and more together), so that the
// lanes of a warp filter chains of about the same length from about the same row and leave the
// chain at about the same time.  One block per (event, sector): a counting sort in shared memory.
// The candidates are still written at the chains' own indices, so the order changes no result.
constexpr int FO_ROWS = 16, FO_LEN = 128, FO_KEYS = (MAX_ROWS / FO_ROWS) * FO_LEN;
__global__ void __launch_bounds__(256) k_follow_order(Work W, int32_t *perm) {
    __shared__ int s_cnt[FO_KEYS];
    const int nr = W.geom->n_rows, ns = W.geom->n_sectors;
    int n_chains = W.counters[CNT_NCHAINS];
    if (n_chains > W.cap_chains) n_chains = W.cap_chains;
    const int nkeys = ((nr + FO_ROWS - 1) / FO_ROWS) * FO_LEN;
    for (int it = blockIdx.x; it < W.n_events * ns; it += gridDim.x) {
        const int b0 = it * nr;
        const int t0 = min(W.chain_off[b0], n_chains), t1 = min(W.chain_off[b0 + nr], n_chains);
        if (t1 <= t0) continue;      // the same for the whole block
        for (int k = threadIdx.x; k < nkeys; k += blockDim.x) s_cnt[k] = 0;
        __syncthreads();
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
            const int key = ((W.chain_bin[t] - b0) / FO_ROWS) * FO_LEN + (FO_LEN - 1 - min(W.chain_len[t], FO_LEN - 1));
            atomicAdd(&s_cnt[key], 1);
        }
        __syncthreads();
        if (threadIdx.x < 32) {      // exclusive scan of the counts by one warp, in key order
            int run = t0;
            for (int k0 = 0; k0 < nkeys; k0 += 32) {
                const int k = k0 + threadIdx.x;
                const int v = k < nkeys ? s_cnt[k] : 0;
                int x = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (threadIdx.x >= o) x += y;
                }
                if (k < nkeys) s_cnt[k] = run + x - v;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
        }
        __syncthreads();
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
            const int key = ((W.chain_bin[t] - b0) / FO_ROWS) * FO_LEN + (FO_LEN - 1 - min(W.chain_len[t], FO_LEN - 1));
            perm[atomicAdd(&s_cnt[key], 1)] = t;
        }
        __syncthreads();
    }
}

// Each warp takes 32 x chunk chains at a time from the queue (no CTA barrier: a warp whose chains
// end early takes the next ones while the others still follow theirs).  SKIP: chains may skip a
// row (the skip-row rule); the plain instantiation keeps the plain reading's registers.
template <bool SKIP>
__global__ void __launch_bounds__(128) k_follow(Work W, const int32_t *perm) {
    const DevGeom &g = *W.geom;
    const int nr = g.n_rows;
    const int lane = threadIdx.x & 31;
    int n_chains = W.counters[CNT_NCHAINS];
    if (n_chains > W.cap_chains) n_chains = W.cap_chains;
    const int chunk = 32 * (W.tune.chunk[3] > 0 ? W.tune.chunk[3] : 1);
    int32_t *q = W.counters + CNT_Q0 + 3;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(q, chunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_chains) break;
        for (int q = base + lane; q < base + chunk && q < n_chains; q += 32) {
            const int t = perm[q];
            const int start = W.chain_start[t], len = W.chain_len[t], bin = W.chain_bin[t];
            const int row0 = bin % nr;
            const int rowbase = bin - row0;
            int32_t *slots = W.cand_slots + (size_t)t * nr;
            Abg fy, fz;
            int row_last;
            if constexpr (!SKIP) {
                // filter along the chain in ascending rows (consecutive rows), writing the chain hits
                int x = start, m0y = 0, m0z = 0;
                for (int k = 0; k < len; k++) {
                    const int y = __ldg(W.pad + x), z = __ldg(W.tim + x);
                    slots[row0 + k] = x;
                    if (k == 0) {
                        m0y = y;
                        m0z = z;
                    } else {
                        if (k == 1) {   // state at the first hit with velocity m1 - m0
                            abg_init(fy, m0y, y, 1);
                            abg_init(fz, m0z, z, 1);
                        }
                        abg_predict(fy);
                        abg_predict(fz);
                        abg_update(fy, y);
                        abg_update(fz, z);
                    }
                    if (k + 1 < len) x = W.up[x];
                }
                row_last = row0 + len - 1;
            } else {
                // the same with links that may skip a row: one filter step per pad row, a skipped
                // row is a prediction without an update and a -1 slot
                int x = start, m0y = 0, m0z = 0, row = row0, rprev = row0;
                for (int k = 0; k < len; k++) {
                    const int y = __ldg(W.pad + x), z = __ldg(W.tim + x);
                    slots[row] = x;
                    const int d = row - rprev;
                    if (k == 0) {
                        m0y = y;
                        m0z = z;
                    } else {
                        if (k == 1) {
                            abg_init(fy, m0y, y, d);
                            abg_init(fz, m0z, z, d);
                        }
                        for (int j = 0; j < d; j++) {
                            abg_predict(fy);
                            abg_predict(fz);
                        }
                        abg_update(fy, y);
                        abg_update(fz, z);
                    }
                    rprev = row;
                    if (k + 1 < len) {
                        x = W.up[x];
                        // the next hit is one row further, or two across a row the link skips
                        if (row + 2 < nr && x >= __ldg(W.bin_off + rowbase + row + 2)) {
                            slots[row + 1] = -1;
                            row += 2;
                        } else {
                            row += 1;
                        }
                    }
                }
                row_last = row;
            }
            int r1, r0;
            const int n_out = extend(W, g, fy, fz, rowbase, row_last, +1, slots, &r1);
            // filter along the chain in descending rows from its last two hits
            if constexpr (!SKIP) {
                const int h1 = slots[row_last], h2 = slots[row_last - 1];
                abg_init(fy, __ldg(W.pad + h1), __ldg(W.pad + h2), 1);
                abg_init(fz, __ldg(W.tim + h1), __ldg(W.tim + h2), 1);
                for (int k = len - 2; k >= 0; k--) {
                    const int h = slots[row0 + k];
                    abg_predict(fy);
                    abg_predict(fz);
                    abg_update(fy, __ldg(W.pad + h));
                    abg_update(fz, __ldg(W.tim + h));
                }
            } else {
                const int h1 = slots[row_last];
                int rp = row_last;
                bool first = true;
                for (int r = row_last - 1; r >= row0; r--) {
                    const int h = slots[r];
                    if (h < 0) continue;
                    const int d = rp - r;
                    if (first) {
                        abg_init(fy, __ldg(W.pad + h1), __ldg(W.pad + h), d);
                        abg_init(fz, __ldg(W.tim + h1), __ldg(W.tim + h), d);
                        first = false;
                    }
                    for (int j = 0; j < d; j++) {
                        abg_predict(fy);
                        abg_predict(fz);
                    }
                    abg_update(fy, __ldg(W.pad + h));
                    abg_update(fz, __ldg(W.tim + h));
                    rp = r;
                }
            }
            const int n_in = extend(W, g, fy, fz, rowbase, row0, -1, slots, &r0);
            W.cand_n[t] = len + n_in + n_out;
            W.cand_rows[t] = r0 | (r1 << 16);
        }
    }
}

}  // namespace

void launch_follow(const Work &W, cudaStream_t s) {
    const int block = W.tune.block[3] > 0 ? W.tune.block[3] : 128;
    const int grid = W.tune.grid[3] > 0 ? W.tune.grid[3] : W.sm_count * 8;
    // the permutation lives in the selection states, which the selection writes before it reads
    int32_t *perm = W.cstate;
    k_follow_order<<<W.sm_count * 8, 256, 0, s>>>(W, perm);
    if (W.rules & TPC_RULE_SKIP_ROW)
        k_follow<true><<<grid, block, 0, s>>>(W, perm);
    else
        k_follow<false><<<grid, block, 0, s>>>(W, perm);
}

}  // namespace tpc
