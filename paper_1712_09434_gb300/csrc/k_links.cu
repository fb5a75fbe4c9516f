// S1 row-bin grid and S2 neighbour finding (cellular automaton, one decision per cluster;
// arxiv 1712.09434 section 3).
//
// S1 (k_grid, one warp per (event, sector, row) bin): clusters of a bin are re-binned into 64 Z
// slabs of 512 LSB by a stable counting sort, so that inside a slab they stay sorted by Y.  The
// payload is packed (Y, Z) int32 plus the row-local index (uint16), stored from a 16-byte aligned
// start pstart(bin).
//
// S2 (k_links, one warp per bin, taken from a work queue): every lane takes one cluster c of row r
// and finds, among u on r+1 and d on r-1 inside the window |dY|, |dZ| <= W_LINK, the pair of
// minimum (D, u, d), D = (Yu+Yd-2Yc)^2 + (Zu+Zd-2Zc)^2 <= D_MAX, all in integers.  The rows are
// read through L1: a CTA-wide staging of rows r+-1 in shared memory by bulk copies was measured
// slower, as the per-bin copy and barriers cost more than the reuse saved.
#include <cstdio>
#include <cstring>

#include "tpc_common.cuh"

namespace tpc {

namespace {

constexpr int LINK_BLOCK = 128;         // threads per CTA of the neighbour finding (at most)
constexpr int LINK_STAGE_CAP = 2048;    // clusters of one row staged in shared memory (staged kernel)
constexpr int LINK_DCAP = 12;           // down-row candidates of a window kept in shared memory

__device__ __forceinline__ int warp_incl(int v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ int slab_of(int z) { int s = z >> ZB_SHIFT; return s < NZB - 1 ? s : NZB - 1; }

__global__ void __launch_bounds__(256) k_grid(Work W) {
    __shared__ int hist[8][NZB];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nw = gridDim.x * (blockDim.x >> 5);
    int *h = hist[wib];
    for (int b = blockIdx.x * (blockDim.x >> 5) + wib; b < W.nbins; b += nw) {
        const int c0 = W.bin_off[b], c1 = W.bin_off[b + 1];
        const int cnt = c1 - c0;
        if (cnt < 0 || cnt > 65535) {
            // row-local indices are 16 bit: flag the bin and give it an empty slab table, so that
            // neighbour searches into it find nothing
            if (lane == 0) set_status(W, ST_BOUNDS);
            for (int i = lane; i <= NZB; i += 32) W.zoff[(size_t)b * ZOFF_STRIDE + i] = 0;
            continue;
        }
        const int ps = pstart_of(c0, b);
        h[lane] = 0;
        h[lane + 32] = 0;
        __syncwarp();
        for (int i = lane; i < cnt; i += 32) atomicAdd(&h[slab_of(W.tim[c0 + i])], 1);
        __syncwarp();
        const int a0 = h[2 * lane], a1 = h[2 * lane + 1];
        const int inc = warp_incl(a0 + a1);
        const int ex = inc - a0 - a1;
        __syncwarp();
        h[2 * lane] = ex;
        h[2 * lane + 1] = ex + a0;
        uint16_t *zo = W.zoff + (size_t)b * ZOFF_STRIDE;
        zo[2 * lane] = (uint16_t)ex;
        zo[2 * lane + 1] = (uint16_t)(ex + a0);
        if (lane == 31) zo[NZB] = (uint16_t)inc;
        __syncwarp();
        // stable scatter in chunks of 32, in cluster (= Y) order
        for (int base = 0; base < cnt; base += 32) {
            const int i = base + lane;
            const bool v = i < cnt;
            int y = 0, z = 0, s = NZB + lane;
            if (v) {
                y = W.pad[c0 + i];
                z = W.tim[c0 + i];
                s = slab_of(z);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, s);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            const int pos = v ? h[s] + rank : 0;
            __syncwarp();
            if (v && rank == 0) h[s] += __popc(peers);
            __syncwarp();
            if (v) {
                W.gyz[ps + pos] = (int32_t)((uint32_t)(y & 0xffff) | ((uint32_t)z << 16));
                W.gloc[ps + pos] = (uint16_t)i;
            }
        }
        __syncwarp();
    }
}

// ---- bulk copy (global -> shared) on an mbarrier, with a bounded wait --------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = SPIN_LIMIT) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

struct RowView {
    const int32_t *yz;        // packed (Y, Z) in slab order
    const uint16_t *loc;      // row-local index
    const uint16_t *zo;       // slab offsets [NZB + 1]
};

__device__ __forceinline__ int lower_y(const int32_t *yz, int lo, int hi, int y) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((int)(int16_t)(yz[mid] & 0xffff) < y) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Whether a row holds a cluster inside the window |dY|, |dZ| <= w around (yc, zc).
__device__ __forceinline__ bool any_in_window(const RowView &rv, int yc, int zc, int w) {
    const int zl = slab_of(max(zc - w, 0)), zh = slab_of(zc + w);
    for (int s = zl; s <= zh; s++) {
        const int hi = rv.zo[s + 1];
        for (int i = lower_y(rv.yz, rv.zo[s], hi, yc - w); i < hi; i++) {
            const int32_t v = rv.yz[i];
            if ((int16_t)(v & 0xffff) > yc + w) break;
            if (abs((int)((uint32_t)v >> 16) - zc) <= w) return true;
        }
    }
    return false;
}

// Warp per row bin, taken from a queue (no CTA barriers: each warp runs at its own pace); the lanes
// take the bin's clusters 32 at a time and read the neighbouring rows' grid data through L1.
// SLAB_ORDER (the default): the lanes take the clusters in the order of the bin's own grid (Z slab,
// then Y), so that the 32 clusters of a warp search the same slabs of rows r+-1 at neighbouring Y
// (12 % faster on the 64-event batch, 23 % on dense time-frame slices); otherwise in cluster
// (Y, Z) order.
template <bool SLAB_ORDER, bool SKIP>
__global__ void __launch_bounds__(LINK_BLOCK) k_links(Work W) {
    // down-row candidates of each lane's cluster: packed (Y, Z) and row-local index, [k][thread]
    __shared__ int32_t s_dv[LINK_DCAP][LINK_BLOCK];
    __shared__ uint16_t s_dl[LINK_DCAP][LINK_BLOCK];
    const DevGeom &g = *W.geom;
    const int nbe = g.n_sectors * g.n_rows;
    const int lane = threadIdx.x & 31;
    int32_t *q = W.counters + CNT_Q0 + 1;
    for (;;) {
        int b = 0;
        if (lane == 0) b = atomicAdd(q, 1);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= W.nbins) break;
        const int r = (b % nbe) % g.n_rows;
        const int c0 = __ldg(W.bin_off + b), c1 = __ldg(W.bin_off + b + 1);
        if (r == 0 || r == g.n_rows - 1) {
            for (int c = c0 + lane; c < c1; c += 32) { W.up[c] = -1; W.down[c] = -1; }
            continue;
        }
        // rows r-1, r+1 and, with the skip-row rule, r-2 and r+2 (where they exist)
        constexpr int NR = SKIP ? 4 : 2;
        RowView rv[NR];
        int cb[NR];
        const bool has2[2] = {SKIP && r >= 2, SKIP && r + 2 <= g.n_rows - 1};
        for (int k = 0; k < NR; k++) {
            const int bb = k == 0 ? b - 1 : k == 1 ? b + 1 : k == 2 ? b - 2 : b + 2;
            if (k >= 2 && !has2[k - 2]) { cb[k] = 0; continue; }
            cb[k] = __ldg(W.bin_off + bb);
            const int ps = pstart_of(cb[k], bb);
            rv[k].yz = W.gyz + ps;
            rv[k].loc = W.gloc + ps;
            rv[k].zo = W.zoff + (size_t)bb * ZOFF_STRIDE;
        }
        const int ps_own = pstart_of(c0, b);
        const bool slab = SLAB_ORDER && c1 - c0 <= 65535;   // larger bins have no grid (flagged)
        for (int i = lane; i < c1 - c0; i += 32) {
            int c, yc, zc;
            if (slab) {
                const int32_t v = W.gyz[ps_own + i];
                c = c0 + W.gloc[ps_own + i];
                yc = (int16_t)(v & 0xffff);
                zc = (int)((uint32_t)v >> 16);
            } else {
                c = c0 + i;
                yc = W.pad[c];
                zc = W.tim[c];
            }
            // each side: the neighbouring row, or (skip-row rule) the row after it with the window
            // doubled when the neighbouring row has no cluster inside the window; fb, fa are the row
            // distances of the down and up partners
            int kd = 0, ku = 1, wd = W_LINK, wu = W_LINK, fb = 1, fa = 1;
            if constexpr (SKIP) {
                if (has2[0] && !any_in_window(rv[0], yc, zc, W_LINK)) { kd = 2; wd = 2 * W_LINK; fb = 2; }
                if (has2[1] && !any_in_window(rv[1], yc, zc, W_LINK)) { ku = 3; wu = 2 * W_LINK; fa = 2; }
            }
            const RowView dv = rv[kd], uv = rv[ku];
            const int kcut = fa * fa + fb * fb + (fa + fb) * (fa + fb);   // 6 for neighbouring rows
            const int zld = slab_of(max(zc - wd, 0)), zhd = slab_of(zc + wd);
            const int zlu = slab_of(max(zc - wu, 0)), zhu = slab_of(zc + wu);
            // down-row candidates inside the window, LINK_DCAP at a time in shared memory; every chunk
            // is compared with all up-row candidates (a window rarely holds more than one chunk).
            // |ey|, |ez| <= 3072, so D fits 32 bits.
            unsigned long long best = ~0ull;
            int nd_all = 0;
            for (int base = 0; base == 0 || base < nd_all; base += LINK_DCAP) {
                int k = 0;
                for (int sd = zld; sd <= zhd; sd++) {
                    const int hd = dv.zo[sd + 1];
                    for (int id = lower_y(dv.yz, dv.zo[sd], hd, yc - wd); id < hd; id++) {
                        const int32_t vd = dv.yz[id];
                        const int yd = (int16_t)(vd & 0xffff);
                        if (yd > yc + wd) break;
                        const int zd = (int)((uint32_t)vd >> 16);
                        if (abs(zd - zc) > wd) continue;
                        if (k >= base && k < base + LINK_DCAP) {
                            s_dv[k - base][threadIdx.x] = vd;
                            s_dl[k - base][threadIdx.x] = dv.loc[id];
                        }
                        k++;
                    }
                }
                nd_all = k;
                const int nd = min(nd_all - base, LINK_DCAP);
                if (nd <= 0) break;
                for (int su = zlu; su <= zhu; su++) {
                    const int hi = uv.zo[su + 1];
                    for (int iu = lower_y(uv.yz, uv.zo[su], hi, yc - wu); iu < hi; iu++) {
                        const int32_t vu = uv.yz[iu];
                        const int yu = (int16_t)(vu & 0xffff);
                        if (yu > yc + wu) break;
                        const int zu = (int)((uint32_t)vu >> 16);
                        if (abs(zu - zc) > wu) continue;
                        const unsigned long long lu = (unsigned long long)uv.loc[iu] << 16;
                        for (int kk = 0; kk < nd; kk++) {
                            const int32_t vd = s_dv[kk][threadIdx.x];
                            const int ey = fb * yu + fa * (int16_t)(vd & 0xffff) - (fa + fb) * yc;
                            const int ez = fb * zu + fa * (int)((uint32_t)vd >> 16) - (fa + fb) * zc;
                            const int D = ey * ey + ez * ez;
                            if (6 * D > kcut * D_MAX) continue;
                            const unsigned long long key = ((unsigned long long)D << 32) | lu | s_dl[kk][threadIdx.x];
                            best = key < best ? key : best;
                        }
                    }
                }
            }
            if (best != ~0ull) {
                W.up[c] = cb[ku] + (int)((best >> 16) & 0xffff);
                W.down[c] = cb[kd] + (int)(best & 0xffff);
            } else {
                W.up[c] = -1;
                W.down[c] = -1;
            }
        }
    }
}

// The same search with rows r-1 and r+1 of every bin staged in shared memory by bulk copies
// (cp.async.bulk on an mbarrier, bounded wait), one CTA per bin, down candidates in registers.
// Selected by tuning (chunk of kernel 1 = 1); measured slower than the L1 version on GB300 (the
// per-bin copy and the CTA barriers cost more than the reuse saves), kept for the autotuner.
__global__ void __launch_bounds__(128) k_links_staged(Work W) {
    extern __shared__ __align__(128) unsigned char smem[];
    int32_t *s_yz[2] = {(int32_t *)smem, (int32_t *)(smem + LINK_STAGE_CAP * 4)};
    uint16_t *s_loc[2] = {(uint16_t *)(smem + 2 * LINK_STAGE_CAP * 4),
                          (uint16_t *)(smem + 2 * LINK_STAGE_CAP * 4 + LINK_STAGE_CAP * 2)};
    __shared__ uint16_t s_zo[2][ZOFF_STRIDE + 1];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_item;
    const DevGeom &g = *W.geom;
    const int nbe = g.n_sectors * g.n_rows;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    int32_t *q = W.counters + CNT_Q0 + 1;
    for (int b = queue_next(q, 1, &s_item); b < W.nbins; b = queue_next(q, 1, &s_item)) {
        const int r = (b % nbe) % g.n_rows;
        const int c0 = W.bin_off[b], c1 = W.bin_off[b + 1];
        if (r == 0 || r == g.n_rows - 1) {
            for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) { W.up[c] = -1; W.down[c] = -1; }
            continue;
        }
        RowView rv[2];
        int nb[2], cb[2];
        bool staged_any = false;
        uint32_t tx = 0;
        for (int k = 0; k < 2; k++) {
            const int bb = k == 0 ? b - 1 : b + 1;          // 0: down row, 1: up row
            cb[k] = W.bin_off[bb];
            nb[k] = W.bin_off[bb + 1] - cb[k];
            const int ps = pstart_of(cb[k], bb);
            for (int i = threadIdx.x; i <= NZB; i += blockDim.x) s_zo[k][i] = W.zoff[(size_t)bb * ZOFF_STRIDE + i];
            rv[k].zo = s_zo[k];
            if (nb[k] > 0 && nb[k] <= LINK_STAGE_CAP) {
                rv[k].yz = s_yz[k];
                rv[k].loc = s_loc[k];
                staged_any = true;
                tx += ((nb[k] * 4 + 15) & ~15) + ((nb[k] * 2 + 15) & ~15);
            } else {
                rv[k].yz = W.gyz + ps;
                rv[k].loc = W.gloc + ps;
            }
        }
        if (staged_any && threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar, tx);
            for (int k = 0; k < 2; k++) {
                if (nb[k] > 0 && nb[k] <= LINK_STAGE_CAP) {
                    const int bb = k == 0 ? b - 1 : b + 1;
                    const int ps = pstart_of(cb[k], bb);
                    bulk_g2s(s_yz[k], W.gyz + ps, (nb[k] * 4 + 15) & ~15, &bar);
                    bulk_g2s(s_loc[k], W.gloc + ps, (nb[k] * 2 + 15) & ~15, &bar);
                }
            }
        }
        __syncthreads();
        if (staged_any) {
            const bool ok = mbar_wait(&bar, phase);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) set_status(W, ST_TIMEOUT);
                mbar_wait(&bar, phase);   // give the copies in flight a second bounded chance
                return;
            }
            phase ^= 1u;
        }
        for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            const int yc = W.pad[c], zc = W.tim[c];
            const int zl = slab_of(max(zc - W_LINK, 0)), zh = slab_of(zc + W_LINK);
            // down-row candidates inside the window, kept in registers (a window holds a few;
            // more than DCAP falls back to rescanning the down row for every up candidate)
            constexpr int DCAP = 8;
            int dyv[DCAP], dzv[DCAP], dlv[DCAP];
            int nd = 0;
            for (int sd = zl; sd <= zh; sd++) {
                const int hd = rv[0].zo[sd + 1];
                for (int id = lower_y(rv[0].yz, rv[0].zo[sd], hd, yc - W_LINK); id < hd; id++) {
                    const int32_t vd = rv[0].yz[id];
                    const int yd = (int16_t)(vd & 0xffff);
                    if (yd > yc + W_LINK) break;
                    const int zd = (int)((uint32_t)vd >> 16);
                    if (abs(zd - zc) > W_LINK) continue;
                    if (nd < DCAP) {
#pragma unroll
                        for (int k = 0; k < DCAP; k++)
                            if (k == nd) { dyv[k] = yd; dzv[k] = zd; dlv[k] = rv[0].loc[id]; }
                    }
                    nd++;
                }
            }
            unsigned long long best = ~0ull;
            if (nd > 0) {
                for (int su = zl; su <= zh; su++) {
                    const int hi = rv[1].zo[su + 1];
                    for (int iu = lower_y(rv[1].yz, rv[1].zo[su], hi, yc - W_LINK); iu < hi; iu++) {
                        const int32_t vu = rv[1].yz[iu];
                        const int yu = (int16_t)(vu & 0xffff);
                        if (yu > yc + W_LINK) break;
                        const int zu = (int)((uint32_t)vu >> 16);
                        if (abs(zu - zc) > W_LINK) continue;
                        const unsigned long long lu = (unsigned long long)rv[1].loc[iu] << 16;
                        if (nd <= DCAP) {
#pragma unroll
                            for (int k = 0; k < DCAP; k++) {
                                if (k < nd) {
                                    const long long ey = yu + dyv[k] - 2 * yc, ez = zu + dzv[k] - 2 * zc;
                                    const long long D = ey * ey + ez * ez;
                                    const unsigned long long key = ((unsigned long long)D << 32) | lu | dlv[k];
                                    if (D <= D_MAX && key < best) best = key;
                                }
                            }
                        } else {
                            for (int sd = zl; sd <= zh; sd++) {
                                const int hd = rv[0].zo[sd + 1];
                                for (int id = lower_y(rv[0].yz, rv[0].zo[sd], hd, yc - W_LINK); id < hd; id++) {
                                    const int32_t vd = rv[0].yz[id];
                                    const int yd = (int16_t)(vd & 0xffff);
                                    if (yd > yc + W_LINK) break;
                                    const int zd = (int)((uint32_t)vd >> 16);
                                    if (abs(zd - zc) > W_LINK) continue;
                                    const long long ey = yu + yd - 2 * yc, ez = zu + zd - 2 * zc;
                                    const long long D = ey * ey + ez * ez;
                                    if (D > D_MAX) continue;
                                    const unsigned long long key = ((unsigned long long)D << 32) | lu | rv[0].loc[id];
                                    best = key < best ? key : best;
                                }
                            }
                        }
                    }
                }
            }
            if (best != ~0ull) {
                W.up[c] = cb[1] + (int)((best >> 16) & 0xffff);
                W.down[c] = cb[0] + (int)(best & 0xffff);
            } else {
                W.up[c] = -1;
                W.down[c] = -1;
            }
        }
        __syncthreads();   // shared rows are overwritten by the next bin's copies
    }
}

}  // namespace

// Bin offsets from the caller are checked before any stage indexes with them: 0 = bin_off[0] <=
// bin_off[1] <= ... <= bin_off[nbins] = n_clusters.  A failing set raises ST_BOUNDS and is
// replaced by one that puts every cluster in the last bin (the outermost row of the last sector,
// which takes no links), so that every later stage stays inside its buffers and finds no tracks.
__global__ void k_bins_check(const int32_t *in, int nbins, int n, int32_t *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nbins; i += gridDim.x * blockDim.x) {
        const int v = in[i];
        bool ok = v >= 0 && v <= n;
        if (i == 0) ok = ok && v == 0;
        if (i == nbins) ok = ok && v == n;
        else ok = ok && v <= in[i + 1];
        if (!ok) atomicOr(bad, 1);
    }
}

__global__ void k_bins_copy(const int32_t *in, int32_t *out, int nbins, int n, const int32_t *bad, int32_t *status) {
    const bool b = *bad != 0;
    if (b && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_BOUNDS);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nbins; i += gridDim.x * blockDim.x)
        out[i] = b ? (i == nbins ? n : 0) : in[i];
}

void launch_bins_check(const Work &W, cudaStream_t s) {
    int grid = (W.nbins + 1 + 255) / 256;
    if (grid > W.sm_count * 4) grid = W.sm_count * 4;
    if (grid < 1) grid = 1;
    k_bins_check<<<grid, 256, 0, s>>>(W.bin_off_in, W.nbins, W.n_clusters, W.counters + CNT_BINS_BAD);
    k_bins_copy<<<grid, 256, 0, s>>>(W.bin_off_in, W.bin_ok, W.nbins, W.n_clusters, W.counters + CNT_BINS_BAD,
                                     W.status);
}

void launch_grid(const Work &W, cudaStream_t s) {
    const int block = W.tune.block[0] > 0 ? W.tune.block[0] : 256;
    const int warps = block / 32;
    int grid = (W.nbins + warps - 1) / warps;
    if (W.tune.grid[0] > 0 && grid > W.tune.grid[0]) grid = W.tune.grid[0];
    if (grid < 1) grid = 1;
    k_grid<<<grid, block, 0, s>>>(W);
}

void prepare_kernels() {
    cudaFuncSetAttribute(k_links_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, LINK_STAGE_CAP * 12);
}

void launch_links(const Work &W, cudaStream_t s) {
    // the staged variant implements the plain reading only: the skip-row rule takes the L1 kernel
    if (W.tune.chunk[1] == 1 && !(W.rules & TPC_RULE_SKIP_ROW)) {     // rows staged in shared memory, CTA per bin
        const int block = W.tune.block[1] > 0 ? W.tune.block[1] : 128;
        int grid = W.tune.grid[1] > 0 ? W.tune.grid[1] : W.sm_count * 8;
        if (grid > W.nbins) grid = W.nbins > 0 ? W.nbins : 1;
        k_links_staged<<<grid, block, (size_t)LINK_STAGE_CAP * 12, s>>>(W);
        return;
    }
    const int block = W.tune.block[1] > 0 ? W.tune.block[1] : 128;
    int grid = W.tune.grid[1] > 0 ? W.tune.grid[1] : W.sm_count * 16;
    const int warps = block / 32;
    if (grid * warps > W.nbins) grid = W.nbins > 0 ? (W.nbins + warps - 1) / warps : 1;
    const bool skip = (W.rules & TPC_RULE_SKIP_ROW) != 0;
    if (W.tune.chunk[1] == 2)       // lanes in cluster (Y, Z) order
        skip ? k_links<false, true><<<grid, block, 0, s>>>(W) : k_links<false, false><<<grid, block, 0, s>>>(W);
    else
        skip ? k_links<true, true><<<grid, block, 0, s>>>(W) : k_links<true, false><<<grid, block, 0, s>>>(W);
}

}  // namespace tpc

// ---- tpc_links_noalloc: grid + neighbour finding without any device allocation ---------------
//
// Some callers cannot allocate device memory when they run: work recorded into a CUDA graph by
// stream capture (cudaMalloc is not a stream operation and cannot be captured), plug-ins hosted
// by a framework whose allocator owns the whole GPU, or real-time code that may only allocate at
// start-up.  For them this entry point runs the same grid and neighbour-finding kernels as the
// tracking path, with their scratch (the Z-slab grid, the work-queue counter, the status word and
// the two geometry numbers the kernels read) in one file-scope device array.  Every GPU that loads
// the library holds that array until the process exits; all calls on a device share it.

namespace tpc {
namespace {

constexpr int NOALLOC_NPAD = TPC_NOALLOC_MAX_CLUSTERS + 8 * (TPC_NOALLOC_MAX_BINS + 2) + 64;
constexpr size_t NOALLOC_OFF_GEOM = 0;                                          // DevGeom
constexpr size_t NOALLOC_OFF_CNT = (sizeof(DevGeom) + 255) & ~(size_t)255;      // counters[64]
constexpr size_t NOALLOC_OFF_BINS = NOALLOC_OFF_CNT + 256;                       // checked bin_off
constexpr size_t NOALLOC_OFF_ZOFF =
    (NOALLOC_OFF_BINS + ((size_t)TPC_NOALLOC_MAX_BINS + 1) * 4 + 255) & ~(size_t)255;
constexpr size_t NOALLOC_OFF_GYZ =
    (NOALLOC_OFF_ZOFF + (size_t)TPC_NOALLOC_MAX_BINS * ZOFF_STRIDE * 2 + 255) & ~(size_t)255;
constexpr size_t NOALLOC_OFF_GLOC = (NOALLOC_OFF_GYZ + (size_t)NOALLOC_NPAD * 4 + 255) & ~(size_t)255;
constexpr size_t NOALLOC_BYTES = (NOALLOC_OFF_GLOC + (size_t)NOALLOC_NPAD * 2 + 255) & ~(size_t)255;

// Writes the geometry numbers the grid and link kernels read, and clears the counters and the
// status word (the array keeps the previous call's contents).
__global__ void k_noalloc_setup(unsigned char *base, int n_sectors, int n_rows) {
    if (threadIdx.x == 0) {
        DevGeom *g = reinterpret_cast<DevGeom *>(base + NOALLOC_OFF_GEOM);
        g->n_sectors = n_sectors;
        g->n_rows = n_rows;
        g->half = n_sectors / 2;
    }
    int32_t *cnt = reinterpret_cast<int32_t *>(base + NOALLOC_OFF_CNT);
    for (int i = threadIdx.x; i < 64; i += blockDim.x) cnt[i] = 0;
}

}  // namespace

}  // namespace tpc

static __device__ __align__(256) unsigned char g_noalloc_scratch[tpc::NOALLOC_BYTES];

#include <mutex>

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_addr[NOALLOC_MAX_DEVICES];   // device address of the array, per device
int g_noalloc_sms[NOALLOC_MAX_DEVICES];

// Once per device, with that device current: the array's device address (its name in host code is
// only a stand-in) and the shared-memory attribute of the link kernel.
int noalloc_setup(int dev, unsigned char **base, int *sms) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            std::fprintf(stderr, "libtpc: tpc_links_noalloc set-up failed: %s\n", cudaGetErrorString(e));
            return TPC_ERR_CUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TPC_ERR_CUDA;
        tpc::prepare_kernels();
        g_noalloc_sms[dev] = n;
        g_noalloc_addr[dev] = static_cast<unsigned char *>(p);
    }
    *base = g_noalloc_addr[dev];
    *sms = g_noalloc_sms[dev];
    return TPC_OK;
}
}  // namespace

extern "C" int tpc_links_noalloc(const tpc_geometry *geom, const tpc_clusters *in, int32_t *up, int32_t *down,
                                 int32_t *status, void *stream) {
    using namespace tpc;
    if (!geom || !in || !in->bin_off || !up || !down || in->n_events < 1 || in->n_clusters < 0 ||
        (in->n_clusters > 0 && (!in->pad_fp || !in->time_fp)) || geom->n_sectors < 2 || geom->n_sectors % 2 ||
        geom->n_sectors > MAX_SECTORS || geom->n_rows < 3 || geom->n_rows > MAX_ROWS)
        return TPC_ERR_INVALID_ARG;
    const long long nbins = (long long)in->n_events * geom->n_sectors * geom->n_rows;
    if (in->n_clusters > TPC_NOALLOC_MAX_CLUSTERS || nbins > TPC_NOALLOC_MAX_BINS) {
        std::fprintf(stderr,
                     "libtpc: tpc_links_noalloc: %d clusters in %lld (event, sector, row) bins exceed the "
                     "static scratch (at most %d clusters and %d bins)\n",
                     in->n_clusters, nbins, TPC_NOALLOC_MAX_CLUSTERS, TPC_NOALLOC_MAX_BINS);
        return TPC_ERR_CAPACITY;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return TPC_ERR_CUDA;
    unsigned char *base = nullptr;
    int sms = 0;
    const int rc = noalloc_setup(dev, &base, &sms);
    if (rc != TPC_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Work W;
    std::memset(&W, 0, sizeof(W));
    W.pad = in->pad_fp;
    W.tim = in->time_fp;
    W.bin_off_in = in->bin_off;
    W.bin_ok = reinterpret_cast<int32_t *>(base + NOALLOC_OFF_BINS);
    W.bin_off = W.bin_ok;
    W.n_events = in->n_events;
    W.n_clusters = in->n_clusters;
    W.nbins = (int)nbins;
    W.ns = geom->n_sectors;
    W.nr = geom->n_rows;
    W.geom = reinterpret_cast<const DevGeom *>(base + NOALLOC_OFF_GEOM);
    W.counters = reinterpret_cast<int32_t *>(base + NOALLOC_OFF_CNT);
    W.status = W.counters + 63;
    W.zoff = reinterpret_cast<uint16_t *>(base + NOALLOC_OFF_ZOFF);
    W.gyz = reinterpret_cast<int32_t *>(base + NOALLOC_OFF_GYZ);
    W.gloc = reinterpret_cast<uint16_t *>(base + NOALLOC_OFF_GLOC);
    W.up = up;
    W.down = down;
    W.sm_count = sms;
    k_noalloc_setup<<<1, 64, 0, s>>>(base, geom->n_sectors, geom->n_rows);
    launch_bins_check(W, s);
    launch_grid(W, s);
    launch_links(W, s);
    if (status) {
        const cudaError_t e = cudaMemcpyAsync(status, W.status, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return TPC_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}

// ---- tpc_selftest_wait_timeout: the bounded-wait failure path, exercised on purpose ------------
namespace tpc {
namespace {
// Waits on an mbarrier that nothing arrives at, with a small iteration limit: the wait gives up,
// the kernel records TPC_ERR_TIMEOUT in *status and returns (no copies in flight, no TMEM held).
__global__ void k_selftest_wait(int32_t *status, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u, limit);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) *status = TPC_ERR_TIMEOUT;
        return;
    }
    if (threadIdx.x == 0) *status = TPC_OK;
}
}  // namespace
}  // namespace tpc

extern "C" int tpc_selftest_wait_timeout(int32_t *status, int32_t spin_limit, void *stream) {
    if (!status || spin_limit < 1 || spin_limit > (1 << 20)) return TPC_ERR_INVALID_ARG;
    tpc::k_selftest_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(status, spin_limit);
    return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}
