// TPC-ITS matching for the drift calibration (arxiv 1712.09434 sections 2.1 and 6: the TPC drift is
// calibrated against tracks of the inner tracker).  Every fitted TPC track (FP32 state and covariance
// at its first hit, in that hit's sector frame) is carried by the exact helix step to x = 0, the
// production vertex, in FP64; an ITS track (global azimuth phi0, z0, tan lambda, q/pT at the vertex
// and their errors) is expressed in the same frame (y = 0, sin phi = sin(phi0 - alpha_k)).  The
// drift calibration is what the match is for, so z only has to fall in a loose window; the match
// chi2 is over (y, sin phi, tan lambda, q/pT) with the TPC covariance plus the ITS errors.  Each side
// keeps its best partner by (floor(chi2 * 2^20), index) (64-bit atomicMin on the ITS side); mutual
// best pairs are matched, and a matched track that starts within the first 8 pad rows, has at least
// 30 hits and |sin phi| < 0.9 at the vertex gets the ITS track's values as its references at the
// vertex (the anchor input of tpc_refit_grad).
#include "kf.cuh"
#include "tpc_common.cuh"

namespace tpc {

namespace {

constexpr int ITS_NPHI = 360;            // azimuth bins of the ITS track grid
constexpr int ITS_NTL = 12;              // tan lambda bins of 0.2 over [-1.2, 1.2) (outside: the end bins)
constexpr int ITS_NBINS = ITS_NPHI * ITS_NTL;
constexpr double ITS_SIGMA_Y = 0.01;     // y of an ITS track at the vertex (cm)
constexpr double ITS_DPHI = 0.1;         // candidate window in azimuth (rad)
constexpr double ITS_DTL = 0.1;          // candidate window in tan lambda
constexpr double ITS_DZ = 2.0;           // candidate window in z at the vertex (cm)
constexpr double ITS_CHI2 = 100.0;       // chi2 gate of a match (loose: see the header)
// references for the calibration only from matched tracks that start at the inner wall, are long
// and stay well inside the local parametrisation at the vertex (the reference reading)
constexpr int REF_MAX_FIRST_ROW = 8;
constexpr int REF_MIN_HITS = 30;
constexpr double REF_MAX_SNP = 0.9;
constexpr double TWO_PI = 6.283185307179586;

// a - 2 pi n with n the nearest integer (IEEE remainder, exact): [-pi, pi]; no loop, so a corrupt
// angle cannot stall the kernel.  |a| <= pi is its own remainder, so that case skips the call.
__device__ __forceinline__ double wrap_pi(double a) { return fabs(a) <= 0.5 * TWO_PI ? a : remainder(a, TWO_PI); }

__device__ __forceinline__ int tl_bin(float tl) {
    const int b = (int)floorf((tl + 1.2f) * 5.0f);
    return b < 0 ? 0 : (b >= ITS_NTL ? ITS_NTL - 1 : b);
}

__device__ __forceinline__ int phi_bin(double phi) {
    int b = (int)floor(phi / TWO_PI * ITS_NPHI);
    b %= ITS_NPHI;
    return b < 0 ? b + ITS_NPHI : b;
}

struct ItsArgs {
    const float *its;          // [n_its][8]
    int n_its;
    int32_t *match_trk, *match_its;
    float *anchor;             // [n_tracks][8] or nullptr
    double kB, alpha0, dalpha; // curvature constant, sector k centre angle = alpha0 + (k mod half) dalpha
    int32_t *cnt, *off, *fill, *list, *sec;   // sec: 1 if the track may carry references
    unsigned long long *best_trk, *best_its;
    double *sc;                // [n_its][2] sin, cos of phi0
};

__global__ void k_its_count(Work W, ItsArgs A) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n_its; i += gridDim.x * blockDim.x) {
        const double phi = A.its[8 * (size_t)i];
        atomicAdd(A.cnt + phi_bin(phi) * ITS_NTL + tl_bin(A.its[8 * (size_t)i + 2]), 1);
        A.sc[2 * (size_t)i] = sin(phi);
        A.sc[2 * (size_t)i + 1] = cos(phi);
        A.best_its[i] = ~0ull;
        A.match_its[i] = -1;
    }
}

__global__ void k_its_fill(Work W, ItsArgs A) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n_its; i += gridDim.x * blockDim.x) {
        const int b = phi_bin(A.its[8 * (size_t)i]) * ITS_NTL + tl_bin(A.its[8 * (size_t)i + 2]);
        A.list[A.off[b] + atomicAdd(A.fill + b, 1)] = i;
    }
}

// chi2 = d^T M^-1 d for a symmetric positive definite 4x4 M (Cholesky); -1 if M is not
__device__ double chi2_4(double M[4][4], const double d[4]) {
    double L[4][4];
    for (int i = 0; i < 4; i++) {
        for (int j = 0; j <= i; j++) {
            double v = M[i][j];
            for (int k = 0; k < j; k++) v -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(v > 0.0)) return -1.0;
                L[i][i] = sqrt(v);
            } else {
                L[i][j] = v / L[j][j];
            }
        }
    }
    double y[4], c2 = 0.0;
    for (int i = 0; i < 4; i++) {
        double v = d[i];
        for (int k = 0; k < i; k++) v -= L[i][k] * y[k];
        y[i] = v / L[i][i];
        c2 += y[i] * y[i];
    }
    return c2;
}

// Thread per TPC track: its state at the vertex, then the ITS tracks of the (azimuth, tan lambda)
// bins that reach into the window; the best (key, ITS index) kept, (key, track) offered to the ITS
// track.
__global__ void k_its_match(Work W, ItsArgs A) {
    const DevGeom &g = *W.geom;
    const int nt = min(*W.n_tracks, W.cap_tracks);
    const int nbe = W.ns * W.nr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        A.best_trk[t] = ~0ull;
        A.sec[t] = -1;
        if (W.ndf[t] <= 0) continue;
        // sector of the first hit: bin of its cluster by binary search in the bin offsets
        const int off = W.trk_off[t];
        const int h = off >= 0 && off < W.cap_hits ? W.trk_hits[off] : -1;
        if (h < 0 || h >= W.n_clusters) {
            set_status(W, ST_BOUNDS);
            continue;
        }
        int lo = 0, hi = W.nbins - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (W.bin_off[mid] <= h) lo = mid; else hi = mid - 1;
        }
        const int k = (lo % nbe) / W.nr;
        const int first_row = lo % W.nr, n_hits = W.trk_off[t + 1] - off;
        kf::State<double> s;
        s.x = W.xref[t];
        s.frame = k;
        s.rref = 0;
        s.yref = s.zref = 0.0;
        for (int i = 0; i < 5; i++) s.p[i] = W.par[5 * (size_t)t + i];
        for (int i = 0, m = 0; i < 5; i++)
            for (int j = 0; j <= i; j++, m++) s.P[i][j] = s.P[j][i] = W.cov[15 * (size_t)t + m];
        if (!kf::prop_fwd<double>(s, -s.x, A.kB, (double)SNP_MAX)) continue;
        A.sec[t] = first_row <= REF_MAX_FIRST_ROW && n_hits >= REF_MIN_HITS && fabs(s.p[2]) < REF_MAX_SNP;
        const double alpha = A.alpha0 + (k % g.half) * A.dalpha;
        const double phi_t = alpha + asin(s.p[2]);
        const double sa = sin(alpha), ca = cos(alpha);
        const float tl32 = (float)s.p[3], z32 = (float)s.p[1];
        // FP32 copies for the pre-checks below
        const float phi32 = (float)phi_t, sa32 = (float)sa, ca32 = (float)ca;
        const float d0_32 = (float)s.p[0], sn32 = (float)s.p[2], q32 = (float)s.p[4];
        const float m0_32 = (float)(s.P[0][0] + ITS_SIGMA_Y * ITS_SIGMA_Y), pss32 = (float)s.P[2][2];
        const float ptt32 = (float)s.P[3][3], pqq32 = (float)s.P[4][4];
        const int ix[4] = {0, 2, 3, 4};
        unsigned long long best = ~0ull;
        const int b0 = (int)floor((phi_t - ITS_DPHI) / TWO_PI * ITS_NPHI), b1 = (int)floor((phi_t + ITS_DPHI) / TWO_PI * ITS_NPHI);
        for (int bb = b0; bb <= b1; bb++) {
            const int bp = ((bb % ITS_NPHI) + ITS_NPHI) % ITS_NPHI;
            // the tan lambda bins that can hold an ITS track within the window (and its margin)
            const int j0 = A.off[bp * ITS_NTL + tl_bin(tl32 - (float)ITS_DTL - 2e-3f)];
            const int j1 = A.off[bp * ITS_NTL + tl_bin(tl32 + (float)ITS_DTL + 2e-3f) + 1];
            for (int j = j0; j < j1; j++) {
                const int i = A.list[j];
                const float *r = A.its + 8 * (size_t)i;
                // FP32 pre-checks with a margin that the exact tests below can only narrow
                if (fabsf(r[2] - tl32) > (float)ITS_DTL + 1e-3f || fabsf(r[1] - z32) > (float)ITS_DZ + 1e-3f) continue;
                {
                    // the azimuth window and the one-component chi2 bound below, in FP32 with margins
                    // (1e-3 rad; 0.1 % of the bound) far above FP32 rounding: they only reject pairs
                    // that the FP64 tests reject too
                    float dph = r[0] - phi32;
                    dph -= rintf(dph * (float)(1.0 / TWO_PI)) * (float)TWO_PI;
                    if (fabsf(dph) > (float)ITS_DPHI + 1e-3f) continue;
                    const float s0 = (float)A.sc[2 * (size_t)i], c0 = (float)A.sc[2 * (size_t)i + 1];
                    const float sdp = s0 * ca32 - c0 * sa32, cph = (c0 * ca32 + s0 * sa32) * r[4];
                    const float d1 = sn32 - sdp, d2 = tl32 - r[2], d3 = q32 - r[3];
                    const float g = (float)ITS_CHI2 * 1.001f;
                    if (d0_32 * d0_32 > g * m0_32 || d1 * d1 > g * (pss32 + cph * cph) ||
                        d2 * d2 > g * (ptt32 + r[6] * r[6]) || d3 * d3 > g * (pqq32 + r[7] * r[7]))
                        continue;
                }
                if (fabs(wrap_pi((double)r[0] - phi_t)) > ITS_DPHI) continue;
                if (fabs((double)r[2] - s.p[3]) > ITS_DTL || fabs((double)r[1] - s.p[1]) > ITS_DZ) continue;
                // sin, cos of phi0 - alpha from those of phi0 and alpha (no transcendental per pair)
                const double s0 = A.sc[2 * (size_t)i], c0 = A.sc[2 * (size_t)i + 1];
                const double sdp = s0 * ca - c0 * sa, cdp = c0 * ca + s0 * sa;
                const double d[4] = {s.p[0], s.p[2] - sdp, s.p[3] - (double)r[2], s.p[4] - (double)r[3]};
                const double cph = cdp * (double)r[4];
                const double ev[4] = {ITS_SIGMA_Y * ITS_SIGMA_Y, cph * cph, (double)r[6] * r[6], (double)r[7] * r[7]};
                // d^T M^-1 d >= d_a^2 / M_aa for a positive definite M (Cauchy-Schwarz): one component
                // beyond the gate on its own, with a margin far above the rounding of the
                // factorisation, rejects the pair without it (the same decision)
                bool beyond = false;
                for (int a = 0; a < 4; a++)
                    beyond |= d[a] * d[a] > ITS_CHI2 * (s.P[ix[a]][ix[a]] + ev[a]) * (1.0 + 1e-9);
                if (beyond) continue;
                double M[4][4];
                for (int a = 0; a < 4; a++)
                    for (int c = 0; c < 4; c++) M[a][c] = s.P[ix[a]][ix[c]] + (a == c ? ev[a] : 0.0);
                const double c2 = chi2_4(M, d);
                if (c2 < 0.0 || c2 > ITS_CHI2) continue;
                const unsigned long long q = (unsigned long long)floor(c2 * 1048576.0);
                const unsigned long long kt = (q << 32) | (unsigned)i;
                best = kt < best ? kt : best;
                atomicMin(A.best_its + i, (q << 32) | (unsigned)t);
            }
        }
        A.best_trk[t] = best;
    }
}

__global__ void k_its_link(Work W, ItsArgs A) {
    const int nt = min(*W.n_tracks, W.cap_tracks);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const unsigned long long v = A.best_trk[t];
        int m = -1;
        if (v != ~0ull) {
            const int i = (int)(v & 0xffffffffu);
            if (A.best_its[i] == ((v & 0xffffffff00000000ull) | (unsigned)t)) m = i;
        }
        A.match_trk[t] = m;
        if (m >= 0) A.match_its[m] = t;
        if (A.anchor) {
            float *a = A.anchor + 8 * (size_t)t;
            if (A.sec[t] <= 0) m = -1;       // matched, but not a reference of the calibration
            const float *r = A.its + 8 * (size_t)(m >= 0 ? m : 0);
            a[0] = m >= 0 ? (float)ITS_SIGMA_Y : 0.f;
            a[1] = m >= 0 ? r[1] : 0.f;
            a[2] = m >= 0 ? r[5] : 0.f;
            a[3] = m >= 0 ? r[2] : 0.f;
            a[4] = m >= 0 ? r[6] : 0.f;
            a[5] = m >= 0 ? r[3] : 0.f;
            a[6] = m >= 0 ? r[7] : 0.f;
            a[7] = 0.f;
        }
    }
}

}  // namespace

int its_match_nphi() { return ITS_NBINS; }
int its_constants(double *out) {
    const double v[] = {ITS_SIGMA_Y, ITS_DPHI, ITS_DTL, ITS_DZ, ITS_CHI2};
    for (int i = 0; i < 5; i++) out[i] = v[i];
    return 5;
}

void launch_its_match(const Work &W, const float *its, int n_its, int32_t *match_trk, int32_t *match_its,
                      float *anchor, double kB, double alpha0, double dalpha, cudaStream_t s) {
    ItsArgs A;
    A.its = its;
    A.n_its = n_its;
    A.match_trk = match_trk;
    A.match_its = match_its;
    A.anchor = anchor;
    A.kB = kB;
    A.alpha0 = alpha0;
    A.dalpha = dalpha;
    // workspace of the tracking, free between calls: counts, offsets and fill levels of the azimuth
    // bins, the ITS tracks sorted by bin, the first-hit sector of every track, the best keys
    A.cnt = W.bin_cnt;
    A.off = W.mrg_off;
    A.fill = W.chain_off;
    A.list = W.mrg_list;
    A.sec = W.trk_n;
    A.best_trk = W.gap_bestT;
    A.best_its = W.gap_bestS;
    A.sc = reinterpret_cast<double *>(W.gap_state);   // 6 words per chain slot >= 2 doubles per ITS track
    const int grid = W.sm_count * 4;
    cudaMemsetAsync(A.cnt, 0, sizeof(int32_t) * (ITS_NBINS + 1), s);
    cudaMemsetAsync(A.fill, 0, sizeof(int32_t) * (ITS_NBINS + 1), s);
    k_its_count<<<grid, 256, 0, s>>>(W, A);
    scan_exclusive(A.cnt, A.off, ITS_NBINS, nullptr, nullptr, W.scan_tmp, W.scan_tmp_len, s);
    k_its_fill<<<grid, 256, 0, s>>>(W, A);
    k_its_match<<<grid, 128, 0, s>>>(W, A);
    k_its_link<<<grid, 256, 0, s>>>(W, A);
}

}  // namespace tpc
