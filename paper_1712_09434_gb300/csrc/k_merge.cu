// S7 inter-sector merging (arxiv 1712.09434 section 3: sectors are tracked independently and
// concurrently, and the track segments are merged afterwards) and assembly of the output tracks.
//
// Ends: the first kept hit of a segment, and its outer end = last kept hit plus the kept hit
// MERGE_BACK positions earlier, on integer (Xtab[row], Y, Z).  The outer end of S is rotated into
// an adjacent sector of the same side with Q30 integer constants (floor shifts), extrapolated
// linearly (floor division) to the row of T's first hit and compared there.  Every valid pair
// offers (D, index) to both sides with 64-bit atomicMin; mutual bests are linked S -> T.  A chain
// of links is one track; a cycle is cut in front of its smallest segment.  Track ids are an
// exclusive scan of head flags in segment order (= seed order), so the output order is canonical.
#include "tpc_common.cuh"

namespace tpc {

namespace {

__device__ __forceinline__ uint32_t key_of(int n_rows, int n_hits, int local) {
    return ((uint32_t)(n_rows - n_hits) << 23) | (uint32_t)local;
}

__device__ __forceinline__ int n_chains_of(const Work &W) {
    const int n = W.counters[CNT_NCHAINS];
    return n < W.cap_chains ? n : W.cap_chains;
}

// first candidate index of the (event, sector) of candidate t
__device__ __forceinline__ int sector_base(const Work &W, int t) {
    const int bin = W.chain_bin[t];
    return W.chain_off[bin - bin % W.nr];
}

// ends of accepted segments; reset of the merge arrays
__global__ void k_merge_ends(Work W) {
    const DevGeom &g = *W.geom;
    const int n = n_chains_of(W);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        W.bestT[t] = ~0ull;
        W.bestS[t] = ~0ull;
        W.next[t] = -1;
        W.prev[t] = -1;
        if (W.seg_n[t] < N_MIN) continue;
        const uint32_t key = key_of(W.nr, W.cand_n[t], t - sector_base(W, t));
        const int rr = W.cand_rows[t];
        const int32_t *sl = W.cand_slots + (size_t)t * W.nr;
        int ring_h[MERGE_BACK + 1], ring_r[MERGE_BACK + 1];
        int first = -1, rf = 0, cnt = 0;
        for (int r = rr & 0xffff; r <= (rr >> 16); r++) {
            const int h = sl[r];
            if (h < 0 || W.owner[h] != key) continue;
            if (first < 0) { first = h; rf = r; }
            ring_h[cnt % (MERGE_BACK + 1)] = h;
            ring_r[cnt % (MERGE_BACK + 1)] = r;
            cnt++;
        }
        if (cnt <= MERGE_BACK) { set_status(W, ST_BOUNDS); continue; }
        const int sector = (W.chain_bin[t] % (W.ns * W.nr)) / W.nr;
        const int iL = (cnt - 1) % (MERGE_BACK + 1), iB = (cnt - 1 - MERGE_BACK) % (MERGE_BACK + 1);
        const int hL = ring_h[iL], rL = ring_r[iL], hB = ring_h[iB], rB = ring_r[iB];
        W.inend[t] = make_int4(g.xtab[rf], W.pad[first], W.tim[first], sector);
        atomicMax(W.sec_ymax + W.chain_bin[t] / (W.ns * W.nr) * W.ns + sector, abs((int)W.pad[first]));
        atomicAdd(W.bin_cnt + (W.chain_bin[t] - W.chain_bin[t] % W.nr) + rf, 1);
        W.outend[2 * t] = make_int4(g.xtab[rB], W.pad[hB], W.tim[hB], sector);
        W.outend[2 * t + 1] = make_int4(g.xtab[rL], W.pad[hL], W.tim[hL], 0);
    }
}

// Accepted segments listed per (event, sector, row of the first kept hit): the merge only looks at
// segments whose first row lies inside the extrapolation reach.
__global__ void k_merge_fill(Work W) {
    const int n = n_chains_of(W);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        if (W.seg_n[t] < N_MIN) continue;
        const int4 e = W.inend[t];
        const int bin0 = W.chain_bin[t] - W.chain_bin[t] % W.nr;
        int lo = 0, hi = W.nr - 1;   // row of the first kept hit from its Xtab value
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (W.geom->xtab[mid] < e.x) lo = mid + 1; else hi = mid;
        }
        const int b = bin0 + lo;
        W.mrg_list[W.mrg_off[b] + atomicAdd(W.bin_cnt + b, 1)] = t;
    }
}

// ---- gap merge inside a sector (TPC_RULE_GAP_MERGE) --------------------------------------------
// The integer steady-state filter of the following (alpha-beta-gamma 1/2, 1/8, 1/32, Q16, floor
// shifts) runs over the kept hits of a segment, one step per pad row and an update per kept hit.
struct Abg {
    long long p, v, a;
};
__device__ __forceinline__ void abg_init(Abg &f, long long m0, long long m1, long long drow) {
    f.p = m0 * 65536;
    f.v = floor_div((m1 - m0) * 65536, drow);
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
__device__ __forceinline__ long long q16_round(long long p) { return (p + 32768) >> 16; }
__device__ __forceinline__ bool gap_inside(const DevGeom &g, const Abg &fy, const Abg &fz, int row) {
    const long long py = q16_round(fy.p), pz = q16_round(fz.p);
    const long long av = fy.v < 0 ? -fy.v : fy.v;
    return !((py < 0 ? -py : py) > g.ymax[row] || pz < 0 || pz > g.zmax || av > (long long)V_MAX * 65536);
}

// Backward filter of every accepted segment over its kept hits in descending rows: the state at its
// first kept hit.  Also resets the gap keys.
__global__ void k_gap_back(Work W) {
    const int n = n_chains_of(W);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        W.gap_bestT[t] = ~0ull;
        W.gap_bestS[t] = ~0ull;
        if (W.seg_n[t] < N_MIN) continue;
        const uint32_t key = key_of(W.nr, W.cand_n[t], t - sector_base(W, t));
        const int rr = W.cand_rows[t];
        const int32_t *sl = W.cand_slots + (size_t)t * W.nr;
        Abg fy{}, fz{};
        int k = 0, rprev = 0, h0 = -1;
        for (int r = rr >> 16; r >= (rr & 0xffff); r--) {
            const int h = sl[r];
            if (h < 0 || W.owner[h] != key) continue;
            if (k == 0) {
                h0 = h;
            } else if (k == 1) {
                abg_init(fy, W.pad[h0], W.pad[h], rprev - r);
                abg_init(fz, W.tim[h0], W.tim[h], rprev - r);
                for (int j = rprev - r; j > 0; j--) { abg_predict(fy); abg_predict(fz); }
                abg_update(fy, W.pad[h]);
                abg_update(fz, W.tim[h]);
            } else {
                for (int j = rprev - r; j > 0; j--) { abg_predict(fy); abg_predict(fz); }
                abg_update(fy, W.pad[h]);
                abg_update(fz, W.tim[h]);
            }
            rprev = r;
            k++;
        }
        long long *st = W.gap_state + 6 * (size_t)t;
        st[0] = fy.p; st[1] = fy.v; st[2] = fy.a;
        st[3] = fz.p; st[4] = fz.v; st[5] = fz.a;
    }
}

// Thread per segment S: forward filter over its kept hits, then row by row across the gap; every
// segment T of the same sector whose first kept hit lies k >= M_MISS + 1 rows past S's last kept
// hit is tested both ways; (D, T) kept for S, (D, S) offered to T by 64-bit atomicMin.
__global__ void k_gap_match(Work W) {
    const DevGeom &g = *W.geom;
    const int n = n_chains_of(W);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        if (W.seg_n[s] < N_MIN) continue;
        const uint32_t key = key_of(W.nr, W.cand_n[s], s - sector_base(W, s));
        const int rr = W.cand_rows[s];
        const int32_t *sl = W.cand_slots + (size_t)s * W.nr;
        Abg fy{}, fz{};
        int k = 0, rprev = 0, h0 = -1, hl = -1;
        for (int r = rr & 0xffff; r <= (rr >> 16); r++) {
            const int h = sl[r];
            if (h < 0 || W.owner[h] != key) continue;
            if (k == 0) {
                h0 = h;
            } else {
                if (k == 1) {
                    abg_init(fy, W.pad[h0], W.pad[h], r - rprev);
                    abg_init(fz, W.tim[h0], W.tim[h], r - rprev);
                }
                for (int j = r - rprev; j > 0; j--) { abg_predict(fy); abg_predict(fz); }
                abg_update(fy, W.pad[h]);
                abg_update(fz, W.tim[h]);
            }
            rprev = r;
            hl = h;
            k++;
        }
        const int rs = rprev;
        const long long ys = W.pad[hl], zs = W.tim[hl];
        const int b0 = W.chain_bin[s] - W.chain_bin[s] % W.nr;   // (event, sector) row 0
        unsigned long long best = ~0ull;
        for (int rt = rs + 1; rt < W.nr && rt <= rs + GAP_MAX; rt++) {
            abg_predict(fy);
            abg_predict(fz);
            if (!gap_inside(g, fy, fz, rt)) break;
            if (rt - rs - 1 < M_MISS) continue;
            const long long py = q16_round(fy.p), pz = q16_round(fz.p);
            const long long w = W_F0 + (long long)W_F1 * (rt - rs - 1);
            for (int i = W.mrg_off[b0 + rt]; i < W.mrg_off[b0 + rt + 1]; i++) {
                const int t = W.mrg_list[i];
                if (t == s) continue;
                const int4 e = W.inend[t];
                const long long dy = e.y - py, dz = e.z - pz;
                if (dy > w || dy < -w || dz > w || dz < -w || dy * dy + dz * dz > w * w) continue;
                const long long *st = W.gap_state + 6 * (size_t)t;
                Abg by{st[0], st[1], st[2]}, bz{st[3], st[4], st[5]};
                bool inside = true;
                for (int j = 1; j <= rt - rs && inside; j++) {
                    abg_predict(by);
                    abg_predict(bz);
                    inside = gap_inside(g, by, bz, rt - j);
                }
                if (!inside) continue;
                const long long ey = ys - q16_round(by.p), ez = zs - q16_round(bz.p);
                if (ey > w || ey < -w || ez > w || ez < -w || ey * ey + ez * ez > w * w) continue;
                const unsigned long long D = (unsigned long long)(dy * dy + dz * dz + ey * ey + ez * ez);
                const unsigned long long kT = (D << 32) | (unsigned)t;
                best = kT < best ? kT : best;
                atomicMin(W.gap_bestS + t, (D << 32) | (unsigned)s);
            }
        }
        W.gap_bestT[s] = best;
    }
}

// Mutual best gap pairs become merge links S -> T before the sector merge runs.
__global__ void k_gap_link(Work W) {
    const int n = n_chains_of(W);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const unsigned long long v = W.gap_bestT[s];
        if (v == ~0ull) continue;
        const int t = (int)(v & 0xffffffffu);
        if (W.gap_bestS[t] == ((v & 0xffffffff00000000ull) | (unsigned)s)) {
            W.next[s] = t;
            W.prev[t] = s;
        }
    }
}

// One warp per outer end S: the lanes take the candidate segments T of the reachable rows of both
// adjacent sectors 32 at a time; the warp keeps the minimum (D, T) for S and every valid pair offers
// (D, S) to T with a 64-bit atomicMin.
__global__ void k_merge_match(Work W) {
    const DevGeom &g = *W.geom;
    const int n = n_chains_of(W);
    const int half = W.ns / 2;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const float pitch = (float)(g.xtab[W.nr - 1] - g.xtab[0]) / (float)(W.nr - 1);
    const bool gap = (W.rules & TPC_RULE_GAP_MERGE) != 0;
    for (int s = gw; s < n; s += nw) {
        if (W.seg_n[s] < N_MIN || (gap && W.next[s] >= 0)) continue;   // a gap successor: no outer end
        const int4 p1 = W.outend[2 * s], p2 = W.outend[2 * s + 1];
        const int ks = p1.w;
        const int ev = W.chain_bin[s] / (W.ns * W.nr);
        const int side0 = ks < half ? 0 : half;
        unsigned long long best = ~0ull;
        for (int k = 0; k < 2; k++) {
            const int sgn = k == 0 ? +1 : -1;
            const int kt = side0 + ((ks - side0) + (k == 0 ? 1 : half - 1)) % half;
            if (k == 1 && kt == side0 + ((ks - side0) + 1) % half) break;   // tiny geometries
            const long long X1 = p1.x, Y1 = p1.y, X2 = p2.x, Y2 = p2.y;
            const long long x1 = (X1 * g.c30 + sgn * Y1 * g.s30) >> 30;
            const long long y1 = (-sgn * X1 * g.s30 + Y1 * g.c30) >> 30;
            const long long x2 = (X2 * g.c30 + sgn * Y2 * g.s30) >> 30;
            const long long y2 = (-sgn * X2 * g.s30 + Y2 * g.c30) >> 30;
            const long long dxs = x2 - x1;
            if (dxs <= 0) continue;
            // The extrapolated Y is monotonic in XT, so its range over the reach |XT - x2| <=
            // MERGE_XMAX is that of the two ends.  If the window around it misses the range of the
            // first-hit Y of every segment of sector kt, no T there can match (the usual case: S
            // ends away from the edge that faces kt).
            {
                const long long ya = y1 + floor_div_pos((x2 - MERGE_XMAX - x1) * (y2 - y1), dxs);
                const long long yb = y1 + floor_div_pos((x2 + MERGE_XMAX - x1) * (y2 - y1), dxs);
                const long long ymin = ya < yb ? ya : yb, ymx = ya < yb ? yb : ya;
                const long long bound = W.sec_ymax[ev * W.ns + kt];
                if (ymin - W_MERGE > bound || ymx + W_MERGE < -bound) continue;
            }
            const int b0 = (ev * W.ns + kt) * W.nr;
            // rows whose plane is within MERGE_XMAX of the extrapolation start (one row of margin;
            // the exact test is below)
            int r_lo = (int)floorf((float)(x2 - MERGE_XMAX - g.xtab[0]) / pitch) - 1;
            int r_hi = (int)ceilf((float)(x2 + MERGE_XMAX - g.xtab[0]) / pitch) + 1;
            r_lo = max(r_lo, 0);
            r_hi = min(r_hi, W.nr - 1);
            if (r_lo > r_hi) continue;
            const int i1 = W.mrg_off[b0 + r_hi + 1];
            for (int i = W.mrg_off[b0 + r_lo] + lane; i < i1; i += 32) {
                const int t = W.mrg_list[i];
                if (gap && W.prev[t] >= 0) continue;                 // a gap predecessor: no first segment
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

__global__ void k_merge_link(Work W) {
    const int n = n_chains_of(W);
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

__global__ void k_merge_heads(Work W) {
    const int n = n_chains_of(W);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        int head = 0;
        if (W.seg_n[s] >= N_MIN) {
            if (W.prev[s] < 0) {
                head = 1;
            } else {
                int x = W.prev[s], k = 0;
                while (x >= 0 && x != s && k < MERGE_MAX_WALK) { x = W.prev[x]; k++; }
                if (k >= MERGE_MAX_WALK) {
                    set_status(W, ST_TIMEOUT);
                } else if (x == s) {       // on a cycle: the smallest segment starts the track
                    int m = s, y = W.next[s];
                    k = 0;
                    while (y != s && k < MERGE_MAX_WALK) { m = y < m ? y : m; y = W.next[y]; k++; }
                    head = m == s;
                }
            }
        }
        W.head[s] = head;
    }
}

// hits per track (walk the segment chain from its head)
__global__ void k_track_count(Work W) {
    const int n = n_chains_of(W);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        if (!W.head[s]) continue;
        const int tid = W.head_id[s];
        if (tid >= W.cap_tracks) { set_status(W, ST_CAPACITY); continue; }
        int sum = 0, x = s, k = 0;
        do {
            sum += W.seg_n[x];
            x = W.next[x];
            k++;
        } while (x >= 0 && !W.head[x] && k < MERGE_MAX_WALK);
        W.trk_n[tid] = sum;
        W.trk_head[tid] = s;
    }
}

// One warp per track: the lanes read 32 row slots of a segment at a time and write its kept hits
// in row order (ballot prefix), then move to the next segment of the merge chain.
__global__ void k_track_write(Work W) {
    const int nt = min(W.counters[CNT_NTRACKS], W.cap_tracks);
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int tid = gw; tid < nt; tid += nw) {
        int pos = W.trk_off[tid];
        int x = W.trk_head[tid], k = 0;
        do {
            const uint32_t key = key_of(W.nr, W.cand_n[x], x - sector_base(W, x));
            const int rr = W.cand_rows[x];
            const int32_t *sl = W.cand_slots + (size_t)x * W.nr;
            const int sector = (W.chain_bin[x] % (W.ns * W.nr)) / W.nr;
            for (int r0 = rr & 0xffff; r0 <= (rr >> 16); r0 += 32) {
                const int r = r0 + lane;
                const int h = r <= (rr >> 16) ? sl[r] : -1;
                const bool kept = h >= 0 && W.owner[h] == key;
                const unsigned m = __ballot_sync(0xffffffffu, kept);
                if (kept) {
                    const int p = pos + __popc(m & ((1u << lane) - 1u));
                    if (p < W.cap_hits) {
                        W.trk_hits[p] = h;
                        W.label[h] = tid;
                        W.trk_pack[2 * p] = (int32_t)((uint32_t)(W.pad[h] & 0xffff) | ((uint32_t)W.tim[h] << 16));
                        W.trk_pack[2 * p + 1] = sector | (r << 16);
                    } else {
                        set_status(W, ST_CAPACITY);
                    }
                }
                pos += __popc(m);
            }
            x = W.next[x];
            k++;
        } while (x >= 0 && !W.head[x] && k < MERGE_MAX_WALK);
    }
}

__global__ void k_event_offsets(Work W) {
    const int n = n_chains_of(W);
    const int nbe = W.ns * W.nr;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= W.n_events; e += gridDim.x * blockDim.x) {
        if (e == W.n_events) {
            W.ev_trk_off[e] = W.counters[CNT_NTRACKS];
            *W.n_tracks = W.counters[CNT_NTRACKS];
        } else {
            W.ev_trk_off[e] = W.head_id[min(W.chain_off[e * nbe], n)];
        }
    }
}

}  // namespace

void launch_merge(const Work &W, cudaStream_t s) {
    const int block = W.tune.block[5] > 0 ? W.tune.block[5] : 128;
    const int grid = W.tune.grid[5] > 0 ? W.tune.grid[5] : W.sm_count * 8;
    cudaMemsetAsync(W.bin_cnt, 0, sizeof(int32_t) * (W.nbins + 1), s);
    cudaMemsetAsync(W.sec_ymax, 0, sizeof(int32_t) * (size_t)W.n_events * W.ns, s);
    k_merge_ends<<<grid, block, 0, s>>>(W);
    scan_exclusive(W.bin_cnt, W.mrg_off, W.nbins, nullptr, nullptr, W.scan_tmp, W.scan_tmp_len, s);
    cudaMemsetAsync(W.bin_cnt, 0, sizeof(int32_t) * (W.nbins + 1), s);
    k_merge_fill<<<grid, block, 0, s>>>(W);
    if (W.rules & TPC_RULE_GAP_MERGE) {
        k_gap_back<<<grid, block, 0, s>>>(W);
        k_gap_match<<<grid, block, 0, s>>>(W);
        k_gap_link<<<grid, block, 0, s>>>(W);
    }
    k_merge_match<<<grid, block, 0, s>>>(W);
    k_merge_link<<<grid, block, 0, s>>>(W);
    k_merge_heads<<<grid, block, 0, s>>>(W);
    scan_exclusive(W.head, W.head_id, W.cap_chains, W.counters + CNT_NCHAINS, W.counters + CNT_NTRACKS,
                   W.scan_tmp, W.scan_tmp_len, s);
    k_track_count<<<grid, block, 0, s>>>(W);
    scan_exclusive(W.trk_n, W.trk_off, W.cap_tracks, W.counters + CNT_NTRACKS, W.counters + CNT_NHITS,
                   W.scan_tmp, W.scan_tmp_len, s);
    k_track_write<<<grid, block, 0, s>>>(W);
    k_event_offsets<<<1, 128, 0, s>>>(W);
}

}  // namespace tpc
