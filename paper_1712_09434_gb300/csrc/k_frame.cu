// S11 time-frame slice merge (arxiv 1712.09434 section 3, its outlook for continuous readout: a
// time frame is cut along the drift-time axis, the slices are tracked one by one, and the track
// segments are merged afterwards) and assembly of the frame tracks.
//
// Input: the clusters of n_slices consecutive slices of slice_len LSB of readout time (the layout
// of a batch, bin = (slice, sector, row), slice-local times) and their per-slice tracks (trk_off,
// trk_hits, ev_trk_off in slice order).  Readout time falls outwards along a track (its drift
// length shrinks as |z| grows), so the piece of a track in slice j+1 (S) ends, at its outer end,
// where the piece in slice j (T) begins.  The outer end of S (last hit and the hit MERGE_BACK
// positions earlier, on integer (Xtab[row], Y, Z + slice_len)) is rotated into the frame of T's
// first hit when that lies in an adjacent sector of the same side (Q30 constants, floor shifts),
// extrapolated linearly to T's first row (floor division) and compared there with the merge
// windows.  Every valid pair offers (D, index) to both sides with 64-bit atomicMin; mutual bests
// are linked S -> T.  Links only go from slice j+1 to slice j, so chains have no cycles; a chain
// is one frame track, ordered by the index of its first slice track.
#include "tpc_common.cuh"

namespace tpc {

namespace {

constexpr int FRAME_BLOCK = 128;

__device__ __forceinline__ int frame_n(const Work &W) { return W.counters[CNT_FRAME_N]; }

// bin of cluster c: the last b with bin_off[b] <= c (bins may be empty)
__device__ __forceinline__ int bin_of(const int32_t *bin_off, int nbins, int c) {
    int lo = 0, hi = nbins - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(bin_off + mid) <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// slice of track t: the last j with ev_trk_off[j] <= t
__device__ __forceinline__ int slice_of(const Work &W, int t) {
    int lo = 0, hi = W.n_events - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(W.s_ev_trk_off + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_frame_count_in(Work W) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int n = *W.s_n_tracks;
        if (n < 0 || n > W.cap_chains) {
            set_status(W, ST_CAPACITY);
            n = n < 0 ? 0 : W.cap_chains;
        }
        W.counters[CNT_FRAME_N] = n;
    }
}

// Ends of every slice track; reset of the link arrays; bucket counts per (slice, sector, first row).
__global__ void k_frame_ends(Work W) {
    const DevGeom &g = *W.geom;
    const int n = frame_n(W);
    const int nbe = W.ns * W.nr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        W.bestT[t] = ~0ull;
        W.bestS[t] = ~0ull;
        W.next[t] = -1;
        W.prev[t] = -1;
        W.inend[t] = make_int4(0, 0, 0, -1);
        W.outend[2 * t + 1] = make_int4(0, 0, 0, -1);
        const int o0 = W.s_trk_off[t], o1 = W.s_trk_off[t + 1];
        if (o0 < 0 || o1 < o0 || o1 > W.n_clusters) { set_status(W, ST_BOUNDS); continue; }
        if (o1 == o0) continue;
        const int h0 = W.s_trk_hits[o0];
        const int hL = W.s_trk_hits[o1 - 1];
        if (h0 < 0 || h0 >= W.n_clusters || hL < 0 || hL >= W.n_clusters) { set_status(W, ST_BOUNDS); continue; }
        const int j = slice_of(W, t);
        if (W.tim[h0] >= W.slice_len) set_status(W, ST_BOUNDS);   // a slice-local time past the slice
        const int b0 = bin_of(W.bin_off, W.nbins, h0) % nbe;
        const int r0 = b0 % W.nr, k0 = b0 / W.nr;
        W.inend[t] = make_int4(g.xtab[r0], W.pad[h0], W.tim[h0], k0);
        atomicAdd(W.bin_cnt + j * nbe + b0, 1);
        if (o1 - o0 <= MERGE_BACK || j == 0) continue;
        const int hB = W.s_trk_hits[o1 - 1 - MERGE_BACK];
        if (hB < 0 || hB >= W.n_clusters) { set_status(W, ST_BOUNDS); continue; }
        const int bL = bin_of(W.bin_off, W.nbins, hL) % nbe, bB = bin_of(W.bin_off, W.nbins, hB) % nbe;
        W.outend[2 * t] = make_int4(g.xtab[bB % W.nr], W.pad[hB], W.tim[hB] + W.slice_len, bL / W.nr);
        W.outend[2 * t + 1] = make_int4(g.xtab[bL % W.nr], W.pad[hL], W.tim[hL] + W.slice_len, j);
    }
}

__global__ void k_frame_fill(Work W) {
    const int n = frame_n(W);
    const int nbe = W.ns * W.nr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int4 e = W.inend[t];
        if (e.w < 0) continue;
        int lo = 0, hi = W.nr - 1;   // row of the first hit from its Xtab value
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (W.geom->xtab[mid] < e.x) lo = mid + 1; else hi = mid;
        }
        const int b = slice_of(W, t) * nbe + e.w * W.nr + lo;
        W.mrg_list[W.mrg_off[b] + atomicAdd(W.bin_cnt + b, 1)] = t;
    }
}

// One warp per outer end S: the lanes take the tracks T of slice j-1 whose first hit lies in the
// reachable rows of the same sector and of both adjacent sectors, 32 at a time.
__global__ void k_frame_match(Work W) {
    const DevGeom &g = *W.geom;
    const int n = frame_n(W);
    const int half = W.ns / 2;
    const int nbe = W.ns * W.nr;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const float pitch = (float)(g.xtab[W.nr - 1] - g.xtab[0]) / (float)(W.nr - 1);
    for (int s = gw; s < n; s += nw) {
        const int4 p2 = W.outend[2 * s + 1];
        if (p2.w < 1) continue;                     // no outer end, or slice 0
        const int4 p1 = W.outend[2 * s];
        const int ks = p1.w, js = p2.w;
        const int side0 = ks < half ? 0 : half;
        const int k_next = side0 + ((ks - side0) + 1) % half;
        const int k_prev = side0 + ((ks - side0) + half - 1) % half;
        unsigned long long best = ~0ull;
        for (int c = 0; c < 3; c++) {
            int kt, sgn;
            if (c == 0) { kt = ks; sgn = 0; }
            else if (c == 1) { kt = k_next; sgn = +1; if (kt == ks) continue; }
            else { kt = k_prev; sgn = -1; if (kt == ks || kt == k_next) continue; }
            long long x1 = p1.x, y1 = p1.y, x2 = p2.x, y2 = p2.y;
            if (sgn != 0) {
                const long long X1 = p1.x, Y1 = p1.y, X2 = p2.x, Y2 = p2.y;
                x1 = (X1 * g.c30 + sgn * Y1 * g.s30) >> 30;
                y1 = (-sgn * X1 * g.s30 + Y1 * g.c30) >> 30;
                x2 = (X2 * g.c30 + sgn * Y2 * g.s30) >> 30;
                y2 = (-sgn * X2 * g.s30 + Y2 * g.c30) >> 30;
            }
            const long long dxs = x2 - x1;
            if (dxs <= 0) continue;
            // The extrapolated time is monotonic in XT, so its range over the reach |XT - x2| <=
            // MERGE_XMAX is that of the two ends.  A slice-j track starts at a time in [0, slice_len);
            // if the window around every extrapolated time misses that range, no T can match (the
            // usual case: S is a whole track whose outer end lies far from the slice start).
            {
                const long long za = p1.z + floor_div_pos((x2 - MERGE_XMAX - x1) * (long long)(p2.z - p1.z), dxs);
                const long long zb = p1.z + floor_div_pos((x2 + MERGE_XMAX - x1) * (long long)(p2.z - p1.z), dxs);
                const long long zmin = za < zb ? za : zb, zmax = za < zb ? zb : za;
                if (zmin - W_MERGE > W.slice_len - 1 || zmax + W_MERGE < 0) continue;
            }
            // rows whose plane is within MERGE_XMAX of the extrapolation start (one row of margin;
            // the exact test is below)
            int r_lo = (int)floorf((float)(x2 - MERGE_XMAX - g.xtab[0]) / pitch) - 1;
            int r_hi = (int)ceilf((float)(x2 + MERGE_XMAX - g.xtab[0]) / pitch) + 1;
            r_lo = max(r_lo, 0);
            r_hi = min(r_hi, W.nr - 1);
            if (r_lo > r_hi) continue;
            const int b0 = (js - 1) * nbe + kt * W.nr;
            const int i1 = W.mrg_off[b0 + r_hi + 1];
            for (int i = W.mrg_off[b0 + r_lo] + lane; i < i1; i += 32) {
                const int t = W.mrg_list[i];
                const int4 e = W.inend[t];
                const long long XT = e.x;
                const long long ax = XT - x2;
                if ((ax < 0 ? -ax : ax) > MERGE_XMAX) continue;
                const long long yp = y1 + floor_div_pos((XT - x1) * (y2 - y1), dxs);
                const long long zp = p1.z + floor_div_pos((XT - x1) * (long long)(p2.z - p1.z), dxs);
                const long long dy = e.y - yp, dz = e.z - zp;
                if (dy > W_MERGE || dy < -W_MERGE || dz > W_MERGE || dz < -W_MERGE) continue;
                const unsigned long long D = (unsigned long long)(dy * dy + dz * dz);
                const unsigned long long kT = (D << 32) | (unsigned)t;
                best = kT < best ? kT : best;
                atomicMin(W.bestS + t, (D << 32) | (unsigned)s);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
            best = v < best ? v : best;
        }
        if (lane == 0) W.bestT[s] = best;
    }
}

__global__ void k_frame_link(Work W) {
    const int n = frame_n(W);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const unsigned long long v = W.bestT[s];
        if (v == ~0ull) continue;
        const int t = (int)(v & 0xffffffffu);
        if (W.bestS[t] == ((v & 0xffffffff00000000ull) | (unsigned)s)) {
            W.next[s] = t;
            W.prev[t] = s;
        }
    }
}

__global__ void k_frame_heads(Work W) {
    const int n = frame_n(W);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        W.head[t] = W.prev[t] < 0;
}

// hits per frame track (walk the chain of slice tracks from its head; a chain visits each slice
// at most once)
__global__ void k_frame_count(Work W) {
    const int n = frame_n(W);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        if (!W.head[t]) continue;
        const int fid = W.head_id[t];
        if (fid >= W.cap_tracks) { set_status(W, ST_CAPACITY); continue; }
        int sum = 0, x = t, k = 0;
        do {
            sum += W.s_trk_off[x + 1] - W.s_trk_off[x];
            x = W.next[x];
            k++;
        } while (x >= 0 && k <= W.n_events);
        if (x >= 0) set_status(W, ST_TIMEOUT);
        W.trk_n[fid] = sum;
        W.trk_head[fid] = t;
    }
}

// One warp per frame track: the lanes copy the hits of each slice track of the chain 32 at a time.
__global__ void k_frame_write(Work W) {
    const int nf = min(W.counters[CNT_FRAME_T], W.cap_tracks);
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int fid = gw; fid < nf; fid += nw) {
        int pos = W.trk_off[fid];
        int x = W.trk_head[fid], k = 0;
        do {
            const int o0 = W.s_trk_off[x], o1 = W.s_trk_off[x + 1];
            for (int i = o0 + lane; i < o1; i += 32) {
                const int p = pos + (i - o0);
                const int h = W.s_trk_hits[i];
                if (h < 0 || h >= W.n_clusters) {
                    set_status(W, ST_BOUNDS);
                } else if (p < W.cap_hits) {
                    W.trk_hits[p] = h;
                    W.label[h] = fid;
                } else {
                    set_status(W, ST_CAPACITY);
                }
            }
            pos += o1 - o0;
            x = W.next[x];
            k++;
        } while (x >= 0 && k <= W.n_events);
    }
}

__global__ void k_frame_final(Work W) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int nf = min(W.counters[CNT_FRAME_T], W.cap_tracks);
        if (W.ev_trk_off) {
            W.ev_trk_off[0] = 0;
            W.ev_trk_off[1] = nf;
        }
        *W.n_tracks = nf;
    }
}

}  // namespace

void launch_frame_merge(const Work &W, cudaStream_t s) {
    const int block = FRAME_BLOCK;
    const int grid = W.sm_count * 8;
    const int nbins = W.nbins;
    cudaMemsetAsync(W.counters + CNT_FRAME_N, 0, 4 * sizeof(int32_t), s);
    if (W.n_clusters > 0) cudaMemsetAsync(W.label, 0xff, (size_t)W.n_clusters * sizeof(int32_t), s);
    cudaMemsetAsync(W.bin_cnt, 0, sizeof(int32_t) * (nbins + 1), s);
    k_frame_count_in<<<1, 32, 0, s>>>(W);
    k_frame_ends<<<grid, block, 0, s>>>(W);
    scan_exclusive(W.bin_cnt, W.mrg_off, nbins, nullptr, nullptr, W.scan_tmp, W.scan_tmp_len, s);
    cudaMemsetAsync(W.bin_cnt, 0, sizeof(int32_t) * (nbins + 1), s);
    k_frame_fill<<<grid, block, 0, s>>>(W);
    k_frame_match<<<grid, block, 0, s>>>(W);
    k_frame_link<<<grid, block, 0, s>>>(W);
    k_frame_heads<<<grid, block, 0, s>>>(W);
    scan_exclusive(W.head, W.head_id, W.cap_chains, W.counters + CNT_FRAME_N, W.counters + CNT_FRAME_T,
                   W.scan_tmp, W.scan_tmp_len, s);
    k_frame_count<<<grid, block, 0, s>>>(W);
    scan_exclusive(W.trk_n, W.trk_off, W.cap_tracks, W.counters + CNT_FRAME_T, W.counters + CNT_FRAME_H,
                   W.scan_tmp, W.scan_tmp_len, s);
    k_frame_write<<<grid, block, 0, s>>>(W);
    k_frame_final<<<1, 32, 0, s>>>(W);
}

}  // namespace tpc
