// Looper-leg pairing (arxiv 1712.09434 section 3: track segments are merged after the sector
// tracking; here the two legs of a low-pT looper, which the tracker finds as two tracks).
//
// A particle whose circle stays inside the TPC goes out to the point of its circle farthest from
// the beam and comes back in.  Both legs are fitted outwards in pad-row order, so the returning
// leg's fit has the opposite curvature and tan lambda of the outgoing one and the same circle.
// Thread per fitted track (FP32 state at its first hit, read as FP64): centre of curvature in the
// global frame, radius, and the z the track reaches at the far point of its circle, carried along
// the fitted direction.  Tracks whose circle has radius <= 130 cm and a centre >= 40 cm from the
// beam are bucketed by (event, azimuth of the centre in 10-degree bins); a thread per candidate
// scans its own and both neighbouring bins (two centres within 5 cm of each other and >= 40 cm
// from the beam differ by less than 7.2 degrees in azimuth) for candidates of opposite curvature
// within the gates (centre 5 cm, radius 5 cm, far-point z 8 cm, |tan lambda_a + tan lambda_b| <=
// 0.05) and keeps the best (floor(D 2^20), index), D = dcentre^2 + dR^2 + dz^2; mutual best pairs
// are joined.  D is symmetric in the two tracks, so each thread finds its own best without atomics.
#include "tpc_common.cuh"

namespace tpc {

namespace {

constexpr double LOOP_RMAX = 130.0;   // largest circle radius of a candidate (cm)
constexpr double LOOP_CMIN = 40.0;    // smallest distance of its centre from the beam (cm)
constexpr double LOOP_DC = 5.0;       // gate on the distance of the two centres (cm)
constexpr double LOOP_DR = 5.0;       // gate on the difference of the radii (cm)
constexpr double LOOP_DZ = 8.0;       // gate on the difference of the far-point z (cm)
constexpr double LOOP_DTL = 0.05;     // gate on |tan lambda_a + tan lambda_b|
constexpr int LOOP_NPHI = 36;         // azimuth bins of the centres per event
constexpr int LOOP_REC = 8;           // doubles per candidate record
constexpr double TWO_PI = 6.283185307179586;

struct LoopArgs {
    int32_t *pair, *leg;
    double kB, alpha0, dalpha;
    double *rec;                  // [nt][LOOP_REC]: cx, cy, R, far-point z, tan lambda, curvature sign, side
    float4 *rec32;                // [nt][2]: (cx, cy, R, far-point z), (tan lambda, curvature sign, 0, 0)
    int32_t *key;                 // [nt] event * LOOP_NPHI + azimuth bin, -1 for a track that is no candidate
    int32_t *cnt, *off, *fill, *list;
    unsigned long long *best;     // [nt] (floor(D 2^20) << 32) | partner
    int nt_cap;                   // tracks the scratch holds
};

__device__ __forceinline__ int n_loop_tracks(const Work &W, const LoopArgs &A) {
    int nt = min(*W.n_tracks, W.cap_tracks);
    return nt < A.nt_cap ? nt : A.nt_cap;
}

__global__ void k_loop_prep(Work W, LoopArgs A) {
    const DevGeom &g = *W.geom;
    const int nt = n_loop_tracks(W, A);
    if (blockIdx.x == 0 && threadIdx.x == 0 && min(*W.n_tracks, W.cap_tracks) > A.nt_cap) set_status(W, ST_CAPACITY);
    const int nbe = W.ns * W.nr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        A.key[t] = -1;
        A.best[t] = ~0ull;
        A.pair[t] = -1;
        if (A.leg) A.leg[t] = 0;
        if (W.ndf[t] <= 0) continue;
        const int off = W.trk_off[t];
        const int h = off >= 0 && off < W.cap_hits ? W.trk_hits[off] : -1;
        if (h < 0 || h >= W.n_clusters) {
            set_status(W, ST_BOUNDS);
            continue;
        }
        int lo = 0, hi = W.nbins - 1;      // bin of the first hit: (event, sector, row)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (W.bin_off[mid] <= h) lo = mid; else hi = mid - 1;
        }
        const int ev = lo / nbe, k = (lo % nbe) / W.nr;
        const double y = W.par[5 * (size_t)t], z = W.par[5 * (size_t)t + 1], sp = W.par[5 * (size_t)t + 2];
        const double tl = W.par[5 * (size_t)t + 3], qpt = W.par[5 * (size_t)t + 4], x = W.xref[t];
        if (!(fabs(sp) < 1.0)) continue;
        const double C = A.kB * qpt;
        if (!(fabs(C) * LOOP_RMAX >= 1.0)) continue;
        const double cp = sqrt(1.0 - sp * sp);
        const double lx = x - sp / C, ly = y + cp / C;     // centre: 1/C to the left of the direction
        const double alpha = A.alpha0 + (k % g.half) * A.dalpha;
        const double ca = cos(alpha), sa = sin(alpha);
        const double cx = lx * ca - ly * sa, cy = lx * sa + ly * ca;
        const double rc = sqrt(cx * cx + cy * cy);
        if (!(rc >= LOOP_CMIN)) continue;
        const double R = 1.0 / fabs(C);
        const double hx = x * ca - y * sa, hy = x * sa + y * ca;                  // first hit
        const double fx = cx + R * cx / rc, fy = cy + R * cy / rc;                // far point
        double turn = (atan2(fy - cy, fx - cx) - atan2(hy - cy, hx - cx)) * (C > 0.0 ? 1.0 : -1.0);
        turn = fmod(turn, TWO_PI);
        if (turn < 0.0) turn += TWO_PI;
        double *r = A.rec + (size_t)t * LOOP_REC;
        r[0] = cx;
        r[1] = cy;
        r[2] = R;
        r[3] = z + tl * R * turn;
        r[4] = tl;
        r[5] = C > 0.0 ? 1.0 : -1.0;
        r[6] = k < g.half ? 1.0 : -1.0;
        A.rec32[2 * (size_t)t] = make_float4((float)cx, (float)cy, (float)R, (float)r[3]);
        A.rec32[2 * (size_t)t + 1] = make_float4((float)tl, (float)r[5], 0.f, 0.f);
        int b = (int)floor(atan2(cy, cx) / TWO_PI * LOOP_NPHI);
        b %= LOOP_NPHI;
        if (b < 0) b += LOOP_NPHI;
        A.key[t] = ev * LOOP_NPHI + b;
        atomicAdd(A.cnt + A.key[t], 1);
    }
}

__global__ void k_loop_fill(Work W, LoopArgs A) {
    const int nt = n_loop_tracks(W, A);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const int b = A.key[t];
        if (b >= 0) A.list[A.off[b] + atomicAdd(A.fill + b, 1)] = t;
    }
}

__global__ void k_loop_match(Work W, LoopArgs A) {
    const int nt = n_loop_tracks(W, A);
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nt; a += gridDim.x * blockDim.x) {
        const int key = A.key[a];
        if (key < 0) continue;
        const double *ra = A.rec + (size_t)a * LOOP_REC;
        const double cx = ra[0], cy = ra[1], R = ra[2], zap = ra[3], tl = ra[4], sg = ra[5];
        const float4 fa = A.rec32[2 * (size_t)a], ga = A.rec32[2 * (size_t)a + 1];
        const int e0 = key - key % LOOP_NPHI, b0 = key % LOOP_NPHI;
        unsigned long long best = ~0ull;
        for (int db = -1; db <= 1; db++) {
            const int bin = e0 + (b0 + db + LOOP_NPHI) % LOOP_NPHI;
            for (int j = A.off[bin]; j < A.off[bin + 1]; j++) {
                const int b = A.list[j];
                if (b == a) continue;
                {   // FP32 pre-checks with margins far above FP32 rounding (coordinates up to a few
                    // hundred cm): they only reject pairs that the FP64 tests below reject
                    const float4 fb = A.rec32[2 * (size_t)b], gb = A.rec32[2 * (size_t)b + 1];
                    if (gb.y == ga.y) continue;
                    const float ex = fa.x - fb.x, ey = fa.y - fb.y;
                    if (ex * ex + ey * ey > (float)((LOOP_DC + 1e-2) * (LOOP_DC + 1e-2)) ||
                        fabsf(fa.z - fb.z) > (float)(LOOP_DR + 1e-2) || fabsf(fa.w - fb.w) > (float)(LOOP_DZ + 1e-2) ||
                        fabsf(ga.x + gb.x) > (float)(LOOP_DTL + 1e-4))
                        continue;
                }
                const double *rb = A.rec + (size_t)b * LOOP_REC;
                if (rb[5] == sg) continue;
                const double dx = cx - rb[0], dy = cy - rb[1];
                const double dc2 = dx * dx + dy * dy, dR = R - rb[2], dz = zap - rb[3];
                if (dc2 > LOOP_DC * LOOP_DC || fabs(dR) > LOOP_DR || fabs(dz) > LOOP_DZ) continue;
                if (fabs(tl + rb[4]) > LOOP_DTL) continue;
                const double D = dc2 + dR * dR + dz * dz;
                const unsigned long long k = ((unsigned long long)floor(D * 1048576.0) << 32) | (unsigned)b;
                best = k < best ? k : best;
            }
        }
        A.best[a] = best;
    }
}

__global__ void k_loop_link(Work W, LoopArgs A) {
    const int nt = n_loop_tracks(W, A);
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nt; a += gridDim.x * blockDim.x) {
        const unsigned long long v = A.best[a];
        if (v == ~0ull) continue;
        const int b = (int)(v & 0xffffffffu);
        if (A.best[b] != ((v & 0xffffffff00000000ull) | (unsigned)a)) continue;
        A.pair[a] = b;
        if (A.leg) {   // the outgoing leg: |z| grows outwards (tan lambda times the side sign larger)
            const double ua = A.rec[(size_t)a * LOOP_REC + 4] * A.rec[(size_t)a * LOOP_REC + 6];
            const double ub = A.rec[(size_t)b * LOOP_REC + 4] * A.rec[(size_t)b * LOOP_REC + 6];
            A.leg[a] = (ua > ub || (ua == ub && a < b)) ? 1 : 2;
        }
    }
}

}  // namespace

int loop_nphi() { return LOOP_NPHI; }
int loop_constants(double *out) {
    const double v[] = {LOOP_RMAX, LOOP_CMIN, LOOP_DC, LOOP_DR, LOOP_DZ, LOOP_DTL};
    for (int i = 0; i < 6; i++) out[i] = v[i];
    return 6;
}

void launch_looper_pairs(const Work &W, int32_t *pair, int32_t *leg, double kB, double alpha0, double dalpha,
                         double *rec, int nt_cap, cudaStream_t s) {
    LoopArgs A;
    A.pair = pair;
    A.leg = leg;
    A.kB = kB;
    A.alpha0 = alpha0;
    A.dalpha = dalpha;
    A.rec = rec;
    A.rec32 = reinterpret_cast<float4 *>(rec + (size_t)nt_cap * LOOP_REC);
    A.nt_cap = nt_cap;
    // workspace of the tracking, free between calls: bin counts, offsets, fill levels, the sorted
    // candidate list, the bin key and the best key of every track
    A.cnt = W.bin_cnt;
    A.off = W.mrg_off;
    A.fill = W.chain_off;
    A.list = W.mrg_list;
    A.key = W.trk_n;
    A.best = W.gap_bestT;
    const int nb = W.n_events * LOOP_NPHI;
    const int grid = W.sm_count * 4;
    cudaMemsetAsync(A.cnt, 0, sizeof(int32_t) * (nb + 1), s);
    cudaMemsetAsync(A.fill, 0, sizeof(int32_t) * (nb + 1), s);
    k_loop_prep<<<grid, 128, 0, s>>>(W, A);
    scan_exclusive(A.cnt, A.off, nb, nullptr, nullptr, W.scan_tmp, W.scan_tmp_len, s);
    k_loop_fill<<<grid, 256, 0, s>>>(W, A);
    k_loop_match<<<grid, 128, 0, s>>>(W, A);
    k_loop_link<<<grid, 256, 0, s>>>(W, A);
}

}  // namespace tpc
