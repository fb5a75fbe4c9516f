// S0 cluster transformation, S8 Kalman-filter refit (FP32) and S9 its adjoint with FP64
// cross-track reductions (arxiv 1712.09434 section 3: Kalman-filter fit and the final track
// refit; sections 2 and 6: calibration of the cluster transformation fed back online).
//
// One thread per track (the paper's one-thread-per-track mapping).  The seed is the circle
// through the first, middle and last hit at the nominal calibration, so it does not depend on
// theta; the fit runs from the last hit to the first.  The adjoint's forward pass stores every K-th
// state (checkpoints) and the reverse sweep recomputes each segment's states from its checkpoint
// before walking it backwards; a variant stores the input state of every step instead (coalesced
// by warp chunk, 80 B per hit) and walks them backwards without recomputation (same results, bit
// for bit).  Per-track chi2 and gradient contributions
// (s_vd, and (d_k, a_k) for every sector the track visits) are written as records and summed in
// FP64 in a fixed order (deterministic).
#include "kf.cuh"
#include "tpc_common.cuh"

namespace tpc {

namespace {

constexpr int CK_K = 16;           // steps between checkpoints
constexpr int ST_SLACK = 4096;     // spare steps per lane for the chunk padding of the stored states
constexpr int CK_WORDS = 25;       // x, p[5], P lower triangle[15], frame, rref, yref, zref
constexpr int ST_WORDS = 20;       // p[5], P lower triangle[15] (stored states: the rest from the hits)
constexpr int REC_SEC = 8;         // sector entries per track record
constexpr int REC_WORDS = 2 + 3 * REC_SEC;
constexpr int NPAR_MAX = 1 + 2 * MAX_SECTORS;
constexpr int RED_T = 64;          // tracks per reduction block

// Gradient workspace: checkpoints (MODE 1/2) | state after the last hit per track (MODE 3/4) |
// chunk lengths, offsets and count | stored states (MODE 3/4).
struct CkLayout {
    float *ck;
    float *fin;
    int32_t *cl, *cb, *cn;
    float *st;
    long long cap_steps;   // chunk steps the stored states can hold
};
inline size_t ck_words_old(long long cap_hits, long long cap_tracks) {
    return (size_t)(cap_hits / CK_K + 2 * cap_tracks + 1) * CK_WORDS;
}
inline size_t ck_words_fin(long long cap_tracks) { return (size_t)cap_tracks * CK_WORDS; }
inline size_t ck_words_ints(long long cap_tracks) { return (size_t)(3 * (cap_tracks / 32 + 2) + 8); }
inline size_t ck_words_st(long long cap_hits) { return (size_t)(cap_hits + 32ll * ST_SLACK) * ST_WORDS; }
inline size_t ck_align(size_t w) { return (w + 31) & ~(size_t)31; }
inline CkLayout ck_layout(float *base, long long cap_hits, long long cap_tracks) {
    CkLayout L;
    L.ck = base;
    L.fin = base + ck_align(ck_words_old(cap_hits, cap_tracks));
    const long long nch = cap_tracks / 32 + 2;
    int32_t *ints = reinterpret_cast<int32_t *>(L.fin + ck_align(ck_words_fin(cap_tracks)));
    L.cl = ints;
    L.cb = ints + nch;
    L.cn = ints + 2 * nch;
    L.st = reinterpret_cast<float *>(ints) + ck_align(ck_words_ints(cap_tracks));
    L.cap_steps = (cap_hits + 32ll * ST_SLACK) / 32;
    return L;
}

struct FitGeo {
    kf::Geo<float> g;
};

// Kahan-Babuska compensated summation in FP32.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

__device__ __forceinline__ void load_geo(const DevGeom &G, FitGeo &f) {
    f.g.kB = G.kB;
    f.g.sig2 = SIGMA2;
    f.g.smax = SNP_MAX;
    f.g.cmin = CPHI_MIN;
    f.g.pitch = G.pitch;
    f.g.half = G.half;
    f.g.rot_c = G.rot_cos;
    f.g.rot_s = G.rot_sin;
    f.g.xr = G.xr;
}

struct HitRaw {
    int k, r, Y, Z;
};

__device__ __forceinline__ HitRaw hit_raw(const Work &W, int i) {
    const int2 v = reinterpret_cast<const int2 *>(W.trk_pack)[i];
    HitRaw h;
    h.Y = (int16_t)(v.x & 0xffff);
    h.Z = (int)((uint32_t)v.x >> 16);
    h.k = v.y & 0xffff;
    h.r = (int)((uint32_t)v.y >> 16);
    return h;
}

// S0: hit under theta (th[0] = 1 - s_vd, th[1+k] = d_k, th[1+ns+k] = a_k) as the filter sees it.
// The kernels take 1 - s_vd from the double theta before rounding to float, so that the drift
// scale keeps its full precision (s_vd itself rounds to 6e-8, a shift that the vertex references
// would notice):
// nominal coordinates (yn = Y*lsb, zn = side*(z_max - D), exact in FP32) plus the calibration
// offsets xl = x_r*a_k*g', yc = y_raw*a_k*g', zc = side*(1 - s_vd)*D + d_k, with the derivative
// factors dzc/ds_vd = -side*D and g' = (rho - x_first)/(span*rho).
// Measurement variances: with model 0 fixed (sigma^2 in y and z); with model 1 the raw errors are
// carried through the transformation, vy = sigma^2 jy^2, vz = sigma^2 jz^2 with jy = 1 + a_k g'
// and jz = s_vd (the change of g' across a pad row is neglected).
struct HitT {
    kf::FHit<float> f;
    float dzds, gp, xr, yraw, jy, jz;
};

__device__ __forceinline__ HitT transform(const DevGeom &G, const float *th, int ns, const HitRaw &h,
                                          int model = 0) {
    HitT o;
    const float side = h.k < G.half ? 1.f : -1.f;
    o.xr = G.xr[h.r];
    o.yraw = (float)h.Y * G.lsb;
    const float D = (float)h.Z * G.lsb;
    o.f.k = h.k;
    o.f.r = h.r;
    o.f.yn = o.yraw;
    o.f.zn = side * (G.z_max - D);
    o.f.zc = side * (th[0] * D) + th[1 + h.k];
    o.dzds = -side * D;
    const float rho = sqrtf(o.xr * o.xr + o.yraw * o.yraw);
    o.gp = (rho - G.x_first) * G.inv_span / rho;
    const float corr = th[1 + ns + h.k] * o.gp;
    o.f.xl = o.xr * corr;
    o.f.yc = o.yraw * corr;
    o.jy = 1.f + corr;
    o.jz = 1.f - th[0];
    o.f.vy = model == 1 ? SIGMA2 * o.jy * o.jy : SIGMA2;
    o.f.vz = model == 1 ? SIGMA2 * o.jz * o.jz : SIGMA2;
    return o;
}

// nominal hit, relative to the last hit E: (x - x_E, y) in E's frame
__device__ __forceinline__ void nominal_rel(const DevGeom &G, const HitRaw &h, const HitRaw &e, float &x, float &y) {
    const float yr = (float)h.Y * G.lsb;
    if (h.k == e.k) {
        x = (float)(h.r - e.r) * G.pitch;
        y = yr;
    } else {   // (x_e, y_e) = R(alpha_h - alpha_e) (x_h, y_h)
        const int m = kf::rot_index(h.k, e.k, G.half);
        const float c = G.rot_cos[m], s = G.rot_sin[m], xh = G.xr[h.r];
        x = xh * c - yr * s - G.xr[e.r];
        y = xh * s + yr * c;
    }
}
__device__ __forceinline__ float nominal_z(const DevGeom &G, const HitRaw &h) {
    const float side = h.k < G.half ? 1.f : -1.f;
    return side * (G.z_max - (float)h.Z * G.lsb);
}

// Prior covariance of the seed: sigma = 1 cm (y, z), 0.1 (sin phi, tan lambda), 1 c/GeV (q/pT).
__device__ __constant__ const float C0[5] = {1.f, 1.f, 0.01f, 0.01f, 1.f};
__device__ __constant__ const float SQRT_C0[5] = {1.f, 1.f, 0.1f, 0.1f, 1.f};

// Seed: sin phi, tan lambda, q/pT from the circle through the nominal first, middle and last hit
// (theta-independent); position = the last hit under theta; references = the last hit.  The caller
// sets the prior covariance.
template <class St>
__device__ bool seed_track(const Work &W, const DevGeom &G, const float *th, int off, int n, St &s) {
    const HitRaw e = hit_raw(W, off + n - 1), a = hit_raw(W, off), b = hit_raw(W, off + (n - 1) / 2);
    float ax, ay, bx, by, ex, ey;
    nominal_rel(G, a, e, ax, ay);
    nominal_rel(G, b, e, bx, by);
    nominal_rel(G, e, e, ex, ey);
    const float ze = nominal_z(G, e);
    if (!kf::seed3<float>(ax, ay, nominal_z(G, a) - ze, bx, by, ex, ey, 0.f, G.kB, SNP_MAX, s.p)) return false;
    const HitT he = transform(G, th, W.ns, e);
    s.p[0] = he.f.yc;
    s.p[1] = he.f.zc;
    s.x = he.f.xl;
    s.rref = e.r;
    s.yref = he.f.yn;
    s.zref = he.f.zn;
    s.frame = e.k;
    return true;
}

__device__ __forceinline__ int n_tracks_of(const Work &W) {
    const int n = W.counters[CNT_NTRACKS];
    return n < W.cap_tracks ? n : W.cap_tracks;
}

// S8 at the nominal calibration: parameters, covariance, chi2, ndf of every track.
// Tracks taken in the order of `order` (decreasing length) when given, so that the lanes of a warp
// fit tracks of about the same length.  Eight blocks a multiprocessor cap it at 64 registers a
// thread (a few spilled words): more resident warps hide the latency of the filter's FMA chain.
__global__ void __launch_bounds__(128, 8) k_refit(Work W, const float *theta, const int32_t *order) {
    __shared__ float th[NPAR_MAX];
    const DevGeom &G = *W.geom;
    const int ns = W.ns, np = 1 + 2 * ns;
    for (int i = threadIdx.x; i < np; i += blockDim.x) th[i] = i == 0 ? 1.f - theta[0] : theta[i];
    __syncthreads();
    FitGeo fg;
    load_geo(G, fg);
    const int nt = n_tracks_of(W);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
        const int t = order ? order[i] : i;
        const int off = W.trk_off[t];
        int n = W.trk_off[t + 1] - off;
        if (off < 0 || n < 0 || off + n > W.cap_hits) {   // hits beyond the packed range: not fitted
            set_status(W, ST_CAPACITY);
            n = 0;
        }
        kf::SqrtState<float> s;
        s.x = 0.f;
        s.rref = 0;
        s.frame = 0;
        s.yref = s.zref = 0.f;
        for (int i = 0; i < 5; i++)
            for (int j = 0; j < 5; j++) s.S[i][j] = i == j ? SQRT_C0[i] : 0.f;
        float chi2 = 0.f;
        bool ok = n >= 3 && seed_track(W, G, th, off, n, s);
        HitRaw nxt = n >= 3 ? hit_raw(W, off + n - 1) : HitRaw{};
        for (int i = n - 1; ok && i >= 0; i--) {
            const HitRaw cur = nxt;
            if (i > 0) nxt = hit_raw(W, off + i - 1);      // next hit's load in flight during this step
            const HitT m = transform(G, th, ns, cur);
            ok = kf::sqrt_step(s, m.f, fg.g, chi2);
        }
        s.p[0] += s.yref;
        s.p[1] += s.zref;
        const float xabs = ok ? G.xr[s.rref] + s.x : 0.f;   // rref is valid only for a seeded track
        for (int i = 0; i < 5; i++) W.par[5 * t + i] = ok ? s.p[i] : 0.f;
        int m = 0;
        for (int i = 0; i < 5; i++)
            for (int j = 0; j <= i; j++) {
                float v = 0.f;
                for (int k = 0; k < 5; k++) v += s.S[i][k] * s.S[j][k];
                W.cov[15 * t + m++] = ok ? v : 0.f;
            }
        W.xref[t] = ok ? xabs : 0.f;
        W.chi2[t] = ok ? chi2 : 0.f;
        W.ndf[t] = ok ? 2 * n - 5 : 0;
    }
}

// Reference measurements at the vertex of one track (reading of the drift calibration by matching
// TPC tracks to inner-tracker tracks, section 6).  anchor[8t..8t+7] = sigma_v of the vertex point
// (y, z) = (0, 0) at x = 0 in the frame of the first hit's sector, then (z0, sigma), (tan lambda,
// sigma), (q/pT, sigma) of the reference track; a sigma <= 0 leaves its term out.  After the last
// hit the state takes the exact helix step to x = 0 (stage 0) and is updated with each term
// (stages 1-4); a failed step fails the track.
struct Anchor {
    float sv, z0, sz, tl, st, q, sq;
    __device__ __forceinline__ bool any() const { return sv > 0.f || sz > 0.f || st > 0.f || sq > 0.f; }
    __device__ __forceinline__ bool fixes_z() const { return sv > 0.f || sz > 0.f; }
};
constexpr int N_ANCHOR_STAGES = 5;

__device__ __forceinline__ Anchor load_anchor(const float *anchor, int t) {
    const float4 a = reinterpret_cast<const float4 *>(anchor)[2 * t];
    const float4 b = reinterpret_cast<const float4 *>(anchor)[2 * t + 1];
    Anchor A;
    A.sv = a.x;
    A.z0 = a.y;
    A.sz = a.z;
    A.tl = a.w;
    A.st = b.x;
    A.q = b.y;
    A.sq = b.z;
    return A;
}

__device__ __forceinline__ bool anchor_fwd(kf::State<float> &s, int j, const Anchor &A, const kf::Geo<float> &g,
                                           float &chi2) {
    switch (j) {
        case 0: {
            const float dx = -(g.xr[s.rref] + s.x);
            if (!kf::prop_fwd(s, dx, g.kB, g.smax, -s.yref, -s.zref)) return false;
            s.x = -g.xr[s.rref];   // absolute x = 0
            s.yref = 0.f;
            s.zref = 0.f;
            return true;
        }
        case 1:
            if (A.sv > 0.f) chi2 += kf::upd_fwd_joseph(s, 0.f, 0.f, A.sv * A.sv, A.sv * A.sv);
            return true;
        case 2:
            if (A.sz > 0.f) chi2 += kf::upd1_fwd(s, 1, A.z0, A.sz * A.sz);
            return true;
        case 3:
            if (A.st > 0.f) chi2 += kf::upd1_fwd(s, 3, A.tl, A.st * A.st);
            return true;
        default:
            if (A.sq > 0.f) chi2 += kf::upd1_fwd(s, 4, A.q, A.sq * A.sq);
            return true;
    }
}

// Adjoint of anchor_fwd stage j; `s` is the state before the stage.
__device__ __forceinline__ void anchor_bwd(const kf::State<float> &s, int j, const Anchor &A,
                                           const kf::Geo<float> &g, kf::Adj<float> &a) {
    switch (j) {
        case 0: {
            const float dx = -(g.xr[s.rref] + s.x);
            const float dxb = kf::prop_bwd(s, dx, g.kB, g.smax, a);
            a.x = -dxb;            // the state's x enters through dx only; the new x is a constant
            return;
        }
        case 1:
            if (A.sv > 0.f) {
                float ymb, zmb, vyb, vzb;
                kf::upd_bwd(s, 0.f, 0.f, A.sv * A.sv, A.sv * A.sv, a, &ymb, &zmb, &vyb, &vzb);
            }
            return;
        case 2:
            if (A.sz > 0.f) kf::upd1_bwd(s, 1, A.z0, A.sz * A.sz, a);
            return;
        case 3:
            if (A.st > 0.f) kf::upd1_bwd(s, 3, A.tl, A.st * A.st, a);
            return;
        default:
            if (A.sq > 0.f) kf::upd1_bwd(s, 4, A.q, A.sq * A.sq, a);
            return;
    }
}

__device__ __forceinline__ void ck_store(float *dst, const kf::State<float> &s) {
    dst[0] = s.x;
    for (int i = 0; i < 5; i++) dst[1 + i] = s.p[i];
    int m = 6;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) dst[m++] = s.P[i][j];
    dst[21] = __int_as_float(s.frame);
    dst[22] = __int_as_float(s.rref);
    dst[23] = s.yref;
    dst[24] = s.zref;
}
__device__ __forceinline__ void ck_load(const float *src, kf::State<float> &s) {
    s.x = src[0];
    for (int i = 0; i < 5; i++) s.p[i] = src[1 + i];
    int m = 6;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) {
            s.P[i][j] = src[m];
            s.P[j][i] = src[m];
            m++;
        }
    s.frame = __float_as_int(src[21]);
    s.rref = __float_as_int(src[22]);
    s.yref = src[23];
    s.zref = src[24];
}

// Stored states (MODE 3/4): the input state of every step, interleaved by warp chunk so that the 32
// lanes of a warp store and load each word with one coalesced access: word k of step q of the
// track at position i of the length order lives at st[((cb[i/32] + q) * ST_WORDS + k) * 32 + i%32].
// Only p and the covariance are stored: the input state of a step is referred to the hit of the
// step before it (x, row, nominal y and z, sector), and that of the first step to its own hit (the
// seed), so the reverse sweep takes them from that hit again.
__device__ __forceinline__ void st_store(float *st, long long step, int lane, const kf::State<float> &s) {
    float *d = st + step * (ST_WORDS * 32) + lane;
    for (int i = 0; i < 5; i++) d[i * 32] = s.p[i];
    int m = 5;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) d[(m++) * 32] = s.P[i][j];
}
__device__ __forceinline__ void st_load(const float *st, long long step, int lane, kf::State<float> &s) {
    const float *d = st + step * (ST_WORDS * 32) + lane;
    for (int i = 0; i < 5; i++) s.p[i] = d[i * 32];
    int m = 5;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) {
            s.P[i][j] = d[m * 32];
            s.P[j][i] = d[m * 32];
            m++;
        }
}

// p and the covariance of a state (20 words; the reference fields are rebuilt from a hit with
// refer_to, as for the stored states)
__device__ __forceinline__ void pp_store(float *d, const kf::State<float> &s) {
    for (int i = 0; i < 5; i++) d[i] = s.p[i];
    int m = 5;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) d[m++] = s.P[i][j];
}
__device__ __forceinline__ void pp_load(const float *d, kf::State<float> &s) {
    for (int i = 0; i < 5; i++) s.p[i] = d[i];
    int m = 5;
    for (int i = 0; i < 5; i++)
        for (int j = 0; j <= i; j++) {
            s.P[i][j] = d[m];
            s.P[j][i] = d[m];
            m++;
        }
}

// S8 + S9: refit under theta; per-track record [chi2, d/ds_vd, (sector, d/dd_k, d/da_k) x 8].
// MODE 0: forward pass only (objective).  Gradient, default: MODE 3 runs the forward pass and stores
// the input state of every step (80 B per hit, coalesced by warp chunk) and the state after the
// last hit (frame -1 marks a track whose fit failed); MODE 4 runs the reverse sweep from the stored
// states.  Gradient with less workspace: MODE 1 stores a checkpoint every CK_K steps, and MODE 2
// recomputes each segment's states from its checkpoint before sweeping it backwards.  Both give
// bit-identical results (the same operations in the same order).  Splitting the forward pass off
// lets it run with fewer registers and more warps than the adjoint.
template <int MODE>
__global__ void __launch_bounds__(128, (MODE == 2 || MODE == 4) ? 4 : (MODE == 0 ? 1 : 7)) k_refit_grad(Work W, const double *theta,
                                                    const float *weight, const float *anchor, int model,
                                                    CkLayout L, float *rec, const int32_t *order) {
    float *ck = L.ck;
    constexpr bool GRAD = MODE != 0;
    __shared__ float th[NPAR_MAX];
    const DevGeom &G = *W.geom;
    const int ns = W.ns, np = 1 + 2 * ns;
    for (int i = threadIdx.x; i < np; i += blockDim.x) th[i] = (float)(i == 0 ? 1.0 - theta[0] : theta[i]);
    __syncthreads();
    FitGeo fg;
    load_geo(G, fg);
    const int nt = n_tracks_of(W);
    __shared__ int s_item;
    int32_t *qh = W.counters + CNT_Q0 + 7;
    for (int base = queue_next(qh, blockDim.x, &s_item); base < nt; base = queue_next(qh, blockDim.x, &s_item)) {
        const int i = base + threadIdx.x;
        if (i >= nt) continue;
        const int t = order[i];
        const int off = W.trk_off[t];
        int n = W.trk_off[t + 1] - off;
        if (off < 0 || n < 0 || off + n > W.cap_hits) {
            set_status(W, ST_CAPACITY);
            n = 0;
        }
        float *r = rec + (size_t)t * REC_WORDS;
        const float w = weight ? weight[t] : 1.f;
        if (w == 0.f) n = 0;   // excluded track: no fit, no adjoint
        // checkpoints of track t: slots [off/CK_K + 2t, ... + ceil(n/CK_K)], the last one the state
        // after the last hit
        float *ckt = ck + ((size_t)(off / CK_K) + 2 * (size_t)t) * CK_WORDS;
        float *ckend = MODE >= 3 ? L.fin + (size_t)t * CK_WORDS
                                 : ckt + (size_t)((n + CK_K - 1) / CK_K) * CK_WORDS;
        const long long step0 = MODE >= 3 ? (long long)L.cb[i >> 5] : 0;    // stored states of this lane
        const int slane = i & 31;
        Anchor A{};
        bool use_anchor = false;
        if (MODE == 0 || MODE == 1 || MODE == 3) {
            kf::State<float> s;
            s.x = 0.f;
            s.rref = 0;
            s.frame = 0;
            s.yref = s.zref = 0.f;
            for (int i = 0; i < 5; i++)
                for (int j = 0; j < 5; j++) s.P[i][j] = i == j ? C0[i] : 0.f;
            float chi2 = 0.f;
            bool ok = n >= 3 && seed_track(W, G, th, off, n, s);
            if (MODE == 3 && ok && step0 + n > L.cap_steps) {   // no room: reported, track dropped
                set_status(W, ST_CAPACITY);
                ok = false;
            }
            HitRaw nxt = n >= 3 ? hit_raw(W, off + n - 1) : HitRaw{};
            for (int q = 0; ok && q < n; q++) {         // processing step q handles hit i = n-1-q
                const HitRaw cur = nxt;
                if (q + 1 < n) nxt = hit_raw(W, off + n - 2 - q);   // next hit's load in flight
                if (MODE == 1 && q % CK_K == 0) ck_store(ckt + (q / CK_K) * CK_WORDS, s);
                if (MODE == 3) st_store(L.st, step0 + q, slane, s);
                const HitT m = transform(G, th, ns, cur, model);
                ok = kf::step_fwd(s, m.f, fg.g, chi2);
            }
            if (GRAD && ok) ck_store(ckend, s);
            use_anchor = anchor != nullptr && ok && (A = load_anchor(anchor, t)).any();
            for (int j = 0; use_anchor && ok && j < N_ANCHOR_STAGES; j++) ok = anchor_fwd(s, j, A, fg.g, chi2);
            if (GRAD && n >= 1 && !ok) ckend[21] = __int_as_float(-1);
            r[0] = ok ? w * chi2 : 0.f;
            r[1] = 0.f;
            for (int k = 0; k < REC_SEC; k++) {
                r[2 + 3 * k] = __int_as_float(-1);
                r[3 + 3 * k] = 0.f;
                r[4 + 3 * k] = 0.f;
            }
            continue;
        }
        // MODE 2 / 4: reverse sweep of a track whose forward pass succeeded
        if (n < 3 || __float_as_int(ckend[21]) < 0) continue;
        use_anchor = anchor != nullptr && (A = load_anchor(anchor, t)).any();
        // reverse sweep from the last hit
        kf::Adj<float> a;
        kf::adj_zero(a);
        Kahan gs, gd, ga;       // compensated FP32 sums over the hits of the track
        int cur_sec = -1, n_ent = 0;
        float ent_d[REC_SEC], ent_a[REC_SEC];
        int ent_s[REC_SEC];
        if (use_anchor) {               // the vertex stages first, each input recomputed from the
            for (int j = N_ANCHOR_STAGES - 1; j >= 0; j--) {   // state after the last hit
                kf::State<float> st;
                ck_load(ckend, st);
                float dummy = 0.f;
                for (int jj = 0; jj < j; jj++) anchor_fwd(st, jj, A, fg.g, dummy);
                anchor_bwd(st, j, A, fg.g, a);
            }
        }
        // one backward step from its input state sin_ (recomputed or stored), then the chain rule
        auto bwd_step = [&](int q, const HitRaw &h, kf::State<float> &sin_) {
            const HitT m = transform(G, th, ns, h, model);
            float xb = 0.f, yb = 0.f, zb = 0.f, vyb = 0.f, vzb = 0.f;
            kf::step_bwd(sin_, m.f, fg.g, a, &xb, &yb, &zb, &vyb, &vzb);
            if (q == 0) {   // the seed position is this hit's (x, y, z)
                xb += a.x;
                yb += a.p[0];
                zb += a.p[1];
            }
            // chain rule through S0
            if (h.k != cur_sec) {
                if (cur_sec >= 0) {
                    if (n_ent < REC_SEC) {
                        ent_s[n_ent] = cur_sec;
                        ent_d[n_ent] = gd.value();
                        ent_a[n_ent] = ga.value();
                    } else {
                        set_status(W, ST_CAPACITY);
                    }
                    n_ent++;
                }
                cur_sec = h.k;
                gd = Kahan();
                ga = Kahan();
            }
            // model 1: vz = sigma^2 s_vd^2, vy = sigma^2 (1 + a_k g')^2
            gs.add(zb * m.dzds + (model == 1 ? vzb * (2.f * SIGMA2) * m.jz : 0.f));
            gd.add(zb);
            ga.add((xb * m.xr + yb * m.yraw + (model == 1 ? vyb * (2.f * SIGMA2) * m.jy : 0.f)) * m.gp);
        };
        if constexpr (MODE == 2) {      // segment by segment from the last checkpoint
            float buf[CK_K * ST_WORDS];     // recomputed step inputs of one segment (p and covariance)
            for (int q0 = ((n - 1) / CK_K) * CK_K; q0 >= 0; q0 -= CK_K) {
                const int q1 = min(q0 + CK_K, n);
                kf::State<float> st;
                ck_load(ckt + (q0 / CK_K) * CK_WORDS, st);
                float dummy = 0.f;
                HitRaw nx = hit_raw(W, off + n - 1 - q0);
                for (int q = q0; q < q1; q++) {
                    const HitRaw cur = nx;
                    if (q + 1 < q1) nx = hit_raw(W, off + n - 2 - q);
                    pp_store(buf + (q - q0) * ST_WORDS, st);
                    const HitT m = transform(G, th, ns, cur, model);
                    kf::step_fwd(st, m.f, fg.g, dummy);
                }
                HitRaw hb = hit_raw(W, off + n - q1);
                for (int q = q1 - 1; q >= q0; q--) {
                    const HitRaw h = hb;
                    if (q > q0) hb = hit_raw(W, off + n - q);
                    kf::State<float> sin_;
                    pp_load(buf + (q - q0) * ST_WORDS, sin_);
                    // the reference of the step's input state: the hit of the step before, or the
                    // seed's own hit for the first step
                    const HitRaw ref = q > q0 ? hb : (q > 0 ? hit_raw(W, off + n - q) : h);
                    const HitT mr = transform(G, th, ns, ref, model);
                    sin_.x = mr.f.xl;
                    sin_.rref = ref.r;
                    sin_.yref = mr.f.yn;
                    sin_.zref = mr.f.zn;
                    sin_.frame = ref.k;
                    bwd_step(q, h, sin_);
                }
            }
        } else {                        // MODE 4: the stored input state of every step
            HitRaw hb = hit_raw(W, off);
            for (int q = n - 1; q >= 0; q--) {
                const HitRaw h = hb;
                if (q > 0) hb = hit_raw(W, off + n - q);
                kf::State<float> sin_;
                st_load(L.st, step0 + q, slane, sin_);
                // the reference of the step's input state: the hit of the step before, or the seed's hit
                const HitRaw &ref = q > 0 ? hb : h;
                const HitT mr = transform(G, th, ns, ref, model);
                sin_.x = mr.f.xl;
                sin_.rref = ref.r;
                sin_.yref = mr.f.yn;
                sin_.zref = mr.f.zn;
                sin_.frame = ref.k;
                bwd_step(q, h, sin_);
            }
        }
        if (cur_sec >= 0) {
            if (n_ent < REC_SEC) {
                ent_s[n_ent] = cur_sec;
                ent_d[n_ent] = gd.value();
                ent_a[n_ent] = ga.value();
            } else {
                set_status(W, ST_CAPACITY);
            }
            n_ent++;
        }
        // Without a z reference at the vertex, a common shift of every z of the track (hits and
        // seed) leaves its chi2 unchanged, so the exact d/dd_k contributions of one track sum to
        // zero.  Project the FP32 sums onto that constraint (equal share of the rounding residual
        // to every entry): a single-sector track contributes exactly zero.
        const int ne = n_ent < REC_SEC ? n_ent : REC_SEC;
        const bool zfree = !(use_anchor && A.fixes_z());
        Kahan tot;
        for (int k = 0; k < ne; k++) tot.add(ent_d[k]);
        const float share = ne > 0 && zfree ? tot.value() / (float)ne : 0.f;
        for (int k = 0; k < ne; k++) {
            r[2 + 3 * k] = __int_as_float(ent_s[k]);
            r[3 + 3 * k] = w * (ne == 1 && zfree ? 0.f : ent_d[k] - share);
            r[4 + 3 * k] = w * ent_a[k];
        }
        r[1] = w * gs.value();
    }
}

// Deterministic FP64 reduction of the track records: block b sums tracks [b*RED_T, (b+1)*RED_T)
// column by column in track order into part[b][np + 1] (column np = chi2); blocks past the last
// track exit at once.
__global__ void __launch_bounds__(RED_T) k_reduce_records(Work W, const float *rec, double *part) {
    __shared__ float m[RED_T][NPAR_MAX + 1];
    const int ns = W.ns, np = 1 + 2 * ns;
    const int nt = n_tracks_of(W);
    if ((long long)blockIdx.x * RED_T >= nt) return;
    const int t = blockIdx.x * RED_T + threadIdx.x;
    for (int j = 0; j <= np; j++) m[threadIdx.x][j] = 0.f;
    if (t < nt) {
        const float *r = rec + (size_t)t * REC_WORDS;
        m[threadIdx.x][np] = r[0];
        m[threadIdx.x][0] = r[1];
        for (int k = 0; k < REC_SEC; k++) {
            const int sec = __float_as_int(r[2 + 3 * k]);
            if (sec < 0 || sec >= ns) continue;
            m[threadIdx.x][1 + sec] += r[3 + 3 * k];
            m[threadIdx.x][1 + ns + sec] += r[4 + 3 * k];
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= np; j += blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < RED_T; i++) acc += (double)m[i][j];
        part[(size_t)blockIdx.x * (np + 1) + j] = acc;
    }
}

// Sum of the block partials: one block per column; thread i takes blocks i, i + 256, ... in order,
// then a fixed tree in shared memory, so the result does not depend on timing.
constexpr int RED_FINAL_T = 256;
__global__ void __launch_bounds__(RED_FINAL_T) k_reduce_final(Work W, int np, const double *part, double *sum_chi2,
                                                             double *grad) {
    __shared__ double acc[RED_FINAL_T];
    const int nt = n_tracks_of(W);
    const int nb = (nt + RED_T - 1) / RED_T;
    const int j = blockIdx.x;
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += RED_FINAL_T) a += part[(size_t)b * (np + 1) + j];
    acc[threadIdx.x] = a;
    __syncthreads();
    for (int w = RED_FINAL_T / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) acc[threadIdx.x] += acc[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (j == np) *sum_chi2 = acc[0];
        else if (grad) grad[j] = acc[0];
    }
}

// Tracks in order of decreasing hit count (counting sort on min(n, LEN_BUCKETS-1)): the adjoint
// takes them from this list, so the 32 tracks of a warp have about the same length and the longest
// ones start first.  The order inside a bucket does not matter (every track is independent).
constexpr int LEN_BUCKETS = 512;

// The lanes of a warp with the same bucket add to it with one atomic (tracks of similar length are
// common, and one atomic per track serialised on the popular buckets).
__global__ void k_len_hist(Work W, int32_t *hist) {
    const int nt = n_tracks_of(W);
    const int lane = threadIdx.x & 31;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const int n = W.trk_off[t + 1] - W.trk_off[t];
        const int b = LEN_BUCKETS - 1 - min(max(n, 0), LEN_BUCKETS - 1);
        const unsigned peers = __match_any_sync(__activemask(), b);
        if (lane == __ffs(peers) - 1) atomicAdd(hist + b, __popc(peers));
    }
}

__global__ void k_len_scan(int32_t *hist) {   // one block of LEN_BUCKETS threads
    __shared__ int sh[LEN_BUCKETS];
    const int i = threadIdx.x;
    sh[i] = hist[i];
    __syncthreads();
    for (int o = 1; o < LEN_BUCKETS; o <<= 1) {
        const int v = i >= o ? sh[i - o] : 0;
        __syncthreads();
        sh[i] += v;
        __syncthreads();
    }
    hist[i] = i > 0 ? sh[i - 1] : 0;          // exclusive offsets
    hist[LEN_BUCKETS + i] = 0;               // fill counters
}

__global__ void k_len_scatter(Work W, int32_t *hist, int32_t *order) {
    const int nt = n_tracks_of(W);
    const int lane = threadIdx.x & 31;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const int n = W.trk_off[t + 1] - W.trk_off[t];
        const int b = LEN_BUCKETS - 1 - min(max(n, 0), LEN_BUCKETS - 1);
        const unsigned peers = __match_any_sync(__activemask(), b);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(hist + LEN_BUCKETS + b, __popc(peers));
        base = __shfl_sync(peers, base, leader);
        order[hist[b] + base + __popc(peers & ((1u << lane) - 1u))] = t;
    }
}

// Longest track of every warp chunk (32 consecutive positions) of the length order, and the
// number of chunks: the chunk offsets of the stored states are their exclusive scan.
__global__ void k_chunk_len(Work W, const int32_t *order, CkLayout L) {
    const int nt = n_tracks_of(W);
    const int nch = (nt + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) *L.cn = nch;
    for (int c = gw; c < nch; c += nw) {
        const int i = 32 * c + lane;
        int len = 0;
        if (i < nt) {
            const int t = order[i];
            len = max(W.trk_off[t + 1] - W.trk_off[t], 0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
        if (lane == 0) L.cl[c] = len;
    }
}

// Bin of every cluster (warp per bin), into a workspace array of N words.
__global__ void k_cluster_bins(Work W, int32_t *cbin) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int b = gw; b < W.nbins; b += nw) {
        const int c0 = __ldg(W.bin_off + b), c1 = __ldg(W.bin_off + b + 1);
        for (int c = max(c0, 0) + lane; c < min(c1, W.n_clusters); c += 32) cbin[c] = b;
    }
}

// Hit list of caller-provided tracks -> packed (Y, Z, sector, row) per hit, the bin of each cluster
// from the map written by k_cluster_bins.
__global__ void k_pack_hits(Work W, const int32_t *cbin) {
    const int nt = n_tracks_of(W);
    int nh = W.trk_off[nt];
    if (nh > W.cap_hits || nh < 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(W, ST_CAPACITY);
        nh = nh < 0 ? 0 : W.cap_hits;
    }
    const int nbe = W.ns * W.nr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nh; i += gridDim.x * blockDim.x) {
        const int h = W.trk_hits[i];
        if (h < 0 || h >= W.n_clusters) {
            set_status(W, ST_BOUNDS);
            W.trk_pack[2 * i] = 0;
            W.trk_pack[2 * i + 1] = 0;
            continue;
        }
        const int lo = cbin[h];
        const int sector = (lo % nbe) / W.nr, row = lo % W.nr;
        W.trk_pack[2 * i] = (int32_t)((uint32_t)(W.pad[h] & 0xffff) | ((uint32_t)W.tim[h] << 16));
        W.trk_pack[2 * i + 1] = sector | (row << 16);
    }
}

}  // namespace

void launch_pack_hits(const Work &W, cudaStream_t s) {
    // the chain-length scratch of the tracking (one word per cluster) holds the cluster -> bin map
    k_cluster_bins<<<W.sm_count * 8, 256, 0, s>>>(W, W.clen);
    k_pack_hits<<<W.sm_count * 4, 256, 0, s>>>(W, W.clen);
}

size_t refit_ck_words(long long cap_hits, long long cap_tracks) {
    return ck_align(ck_words_old(cap_hits, cap_tracks)) + ck_align(ck_words_fin(cap_tracks)) +
           ck_align(ck_words_ints(cap_tracks)) + ck_words_st(cap_hits);
}
int refit_rec_words(int cap_tracks) { return cap_tracks * REC_WORDS; }
int refit_part_doubles(int cap_tracks, int ns) { return ((cap_tracks + RED_T - 1) / RED_T + 1) * (2 * ns + 2); }


void launch_len_order(const Work &W, int32_t *order, int32_t *hist, cudaStream_t s) {
    cudaMemsetAsync(hist, 0, sizeof(int32_t) * LEN_BUCKETS, s);
    k_len_hist<<<W.sm_count * 4, 256, 0, s>>>(W, hist);
    k_len_scan<<<1, LEN_BUCKETS, 0, s>>>(hist);
    k_len_scatter<<<W.sm_count * 4, 256, 0, s>>>(W, hist, order);
}

void launch_refit(const Work &W, const float *theta, const int32_t *order, cudaStream_t s) {
    const int block = W.tune.block[6] > 0 ? W.tune.block[6] : 128;
    const int grid = W.tune.grid[6] > 0 ? W.tune.grid[6] : W.sm_count * 8;
    k_refit<<<grid, block, 0, s>>>(W, theta, order);
}

void launch_refit_grad_fit(const Work &W, const double *theta, const float *weight, const float *anchor, int model,
                           bool grad, float *ck, long long ck_hits, long long ck_tracks, float *rec, int32_t *order,
                           int32_t *hist, bool sorted, cudaStream_t s) {
    const int block = W.tune.block[7] > 0 ? W.tune.block[7] : 128;
    const int grid = W.tune.grid[7] > 0 ? W.tune.grid[7] : W.sm_count * 8;
    const CkLayout L = ck_layout(ck, ck_hits, ck_tracks);
    cudaMemsetAsync(W.counters + CNT_Q0 + 7, 0, sizeof(int32_t), s);
    if (!sorted) launch_len_order(W, order, hist, s);
    if (grad && W.tune.chunk[7] == 1) {     // every step's input state stored, no recomputation
        k_chunk_len<<<W.sm_count * 4, 256, 0, s>>>(W, order, L);
        scan_exclusive(L.cl, L.cb, (int)(ck_tracks / 32 + 1), L.cn, L.cn + 1, W.scan_tmp, W.scan_tmp_len, s);
        k_refit_grad<3><<<grid, block, 0, s>>>(W, theta, weight, anchor, model, L, rec, order);
        cudaMemsetAsync(W.counters + CNT_Q0 + 7, 0, sizeof(int32_t), s);
        k_refit_grad<4><<<grid, block, 0, s>>>(W, theta, weight, anchor, model, L, rec, order);
    } else if (grad) {                      // checkpoints every CK_K steps, states recomputed (default)
        k_refit_grad<1><<<grid, block, 0, s>>>(W, theta, weight, anchor, model, L, rec, order);
        cudaMemsetAsync(W.counters + CNT_Q0 + 7, 0, sizeof(int32_t), s);
        k_refit_grad<2><<<grid, block, 0, s>>>(W, theta, weight, anchor, model, L, rec, order);
    } else {
        k_refit_grad<0><<<grid, block, 0, s>>>(W, theta, weight, anchor, model, L, rec, order);
    }
}

void launch_refit_grad_reduce(const Work &W, double *sum_chi2, double *grad, const float *rec, double *part,
                              cudaStream_t s) {
    const int cap = W.cap_tracks < W.cap_chains ? W.cap_tracks : W.cap_chains;
    const int nb = (cap + RED_T - 1) / RED_T;
    k_reduce_records<<<nb > 0 ? nb : 1, RED_T, 0, s>>>(W, rec, part);
    k_reduce_final<<<2 + 2 * W.ns, RED_FINAL_T, 0, s>>>(W, 1 + 2 * W.ns, part, sum_chi2, grad);
}

}  // namespace tpc
