// Internal definitions shared by the CUDA translation units of libtpc (not part of the ABI).
//
// Reading constants of the integer track finding (arxiv 1712.09434 section 3 fixes only the
// structure: CA seeding, Kalman following, sector merging; these values are this library's
// readings and are declared independently of any other implementation).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tpc.h"

namespace tpc {

constexpr int W_LINK = 384;       // neighbour window |dY|, |dZ| (LSB)
constexpr int D_MAX = 13600;      // max squared second difference of a link triplet (LSB^2)
constexpr int N_SEED = 5;         // minimum chain length kept as a seed
constexpr int M_MISS = 8;         // following stops after this many consecutive empty rows
constexpr int W_F0 = 77;          // following search radius without a miss (LSB)
constexpr int W_F1 = 38;          // radius growth per consecutive miss (LSB)
constexpr int V_MAX = 320;        // following stops when |dY/row| exceeds this (LSB/row)
constexpr int N_MIN = 10;         // minimum kept hits of an accepted segment
constexpr int W_MERGE = 192;      // merge window |dY|, |dZ| (LSB)
constexpr int MERGE_XMAX = 2048;  // maximum merge extrapolation distance (LSB)
constexpr int MERGE_BACK = 3;     // direction baseline of a segment end (hits)
constexpr int GAP_MAX = 24;       // gap merge: largest row distance between the two segment ends

constexpr int MAX_ROWS = 512;
constexpr int MAX_SECTORS = 64;
constexpr int ZB_SHIFT = 9;       // grid Z slab = 512 LSB (4 cm): a +-384 window spans <= 2 slabs
constexpr int NZB = 64;           // slabs per row bin (Z >> 9 clamped to 63)
constexpr int ZOFF_STRIDE = NZB + 1;

constexpr float SIGMA2 = 0.01f;   // measurement variance (cm^2)
constexpr float SNP_MAX = 0.999f; // |sin phi| limit of the local helix state
constexpr float CPHI_MIN = 0.01f; // minimum cos phi after a sector rotation

constexpr uint32_t KEY_NONE = 0xffffffffu;
constexpr int SELECT_MAX_ROUNDS = 1 << 14;
constexpr int MERGE_MAX_WALK = 1 << 12;
constexpr long long SPIN_LIMIT = 1ll << 22;   // bounded waits on mbarriers

// Status bits (device status word); mapped to TPC_ERR_* on the host.
constexpr int ST_CAPACITY = 1;
constexpr int ST_TIMEOUT = 2;
constexpr int ST_BOUNDS = 4;

// Geometry tables, computed on the host in double precision and uploaded once.
struct DevGeom {
    int n_sectors, n_rows, half;
    int zmax;                 // round(z_max / lsb)
    long long c30, s30;       // round(cos, sin(2*half angle) * 2^30)
    float kB;                 // -0.299792458e-2 * Bz
    float lsb, z_max, x_first, inv_span, pitch;
    float xr[MAX_ROWS];       // row plane x [cm]
    int ymax[MAX_ROWS];       // floor(x_r tan(half angle) / lsb)
    int xtab[MAX_ROWS];       // round(x_r / lsb)
    float rot_cos[MAX_SECTORS], rot_sin[MAX_SECTORS];  // cos/sin(m * 2*half angle), m + half
};

// Launch-shape tuning resolved from tpc_tuning (kernel index as in tpc.h).
struct Tune {
    int block[TPC_N_TUNE];
    int grid[TPC_N_TUNE];
    int chunk[TPC_N_TUNE];
};

// Everything a kernel needs: inputs, outputs, workspace.  Passed by value.
struct Work {
    // inputs
    const int16_t *pad;
    const uint16_t *tim;
    const int32_t *bin_off;   // the checked copy of the bin offsets (bin_ok) that every stage reads
    const int32_t *bin_off_in;  // the caller's bin offsets, read only by the check
    int n_events, n_clusters, nbins;
    int ns, nr;               // sectors, rows (host copies of the geometry)
    int rules;                // TPC_RULE_* bits (0: the plain readings)
    // outputs
    int32_t *label, *trk_off, *trk_hits, *ev_trk_off, *ndf, *n_tracks;
    float *par, *xref, *cov, *chi2;
    int cap_tracks, cap_hits;
    // geometry
    const DevGeom *geom;
    // workspace: checked bin offsets [nbins + 1]: the caller's, or (if any offset is out of range
    // or decreasing, or the offsets do not run from 0 to n_clusters) every cluster in the last bin
    int32_t *bin_ok;
    // workspace: grid (S1)
    int32_t *gyz;             // [npad] packed (Y & 0xffff) | (Z << 16), slab order
    uint16_t *gloc;           // [npad] row-local cluster index, slab order
    uint16_t *zoff;           // [nbins * ZOFF_STRIDE] row-local slab offsets
    // links (S2)
    int32_t *up, *down;       // [N]
    // chains (S3, S4)
    int32_t *clen;            // [N] kept chain length at its start cluster, else 0
    int32_t *bin_cnt;         // [nbins + 1] chains starting in the bin
    int32_t *chain_off;       // [nbins + 1] exclusive scan of bin_cnt
    int32_t *chain_start, *chain_len, *chain_bin;   // [cap_chains]
    int cap_chains;
    // following (S5)
    int32_t *cand_n;          // [cap_chains]
    int32_t *cand_rows;       // [cap_chains] row0 | row1 << 16
    int32_t *cand_slots;      // [cap_chains * n_rows] cluster per row inside [row0, row1], else -1
    // selection (S6)
    uint32_t *claim;          // [2N] 64-bit round-tagged claims
    uint32_t *owner;          // [N]  key of the accepted candidate owning the cluster
    int32_t *cstate;          // [cap_chains] selection state
    int32_t *seg_n;           // [cap_chains] kept hits, 0 if rejected
    // merge (S7)
    unsigned long long *bestT, *bestS;  // [cap_chains]
    int32_t *next, *prev;     // [cap_chains]
    int4 *inend;              // [cap_chains] first kept hit (Xtab, Y, Z, sector)
    int32_t *mrg_off;         // [nbins + 1] accepted segments per (event, sector, first row)
    int32_t *mrg_list;        // [cap_chains] segment indices in mrg_off order
    int4 *outend;             // [cap_chains * 2] (X1, Y1, Z1, sector), (X2, Y2, Z2, -) of the outer end
    int32_t *sec_ymax;        // [max_events * n_sectors] largest |Y| of a segment's first kept hit
    int32_t *head;            // [cap_chains] 1 if the segment starts a merged track
    int32_t *head_id;         // [cap_chains + 1] exclusive scan of head = track id
    int32_t *trk_n;           // [cap_tracks + 1] hits per track, then exclusive scan
    int32_t *trk_head;        // [cap_tracks] head segment of each track
    int32_t *trk_pack;        // [cap_hits * 2] (Y | Z<<16, sector | row<<16) per hit
    // gap merge (TPC_RULE_GAP_MERGE)
    long long *gap_state;     // [cap_chains * 6] backward filter state (p, v, a of Y and Z) at the first kept hit
    unsigned long long *gap_bestT, *gap_bestS;  // [cap_chains] (D << 32 | index)
    // time-frame slice merge (S11): the per-slice tracks it reads (device)
    const int32_t *s_trk_off, *s_trk_hits, *s_ev_trk_off, *s_n_tracks;
    int slice_len;
    // scan scratch
    int32_t *scan_tmp;        // [scan_tmp_len]
    int scan_tmp_len;
    // counters and status
    int32_t *counters;        // [64]: see CNT_*
    int32_t *status;          // [1]
    int sm_count;
    Tune tune;
};

enum {
    CNT_NCHAINS = 0,
    CNT_NTRACKS = 1,
    CNT_NHITS = 2,
    CNT_ROUNDS = 3,           // largest number of selection rounds of any sector
    CNT_FRAME_N = 4,          // slice merge: slice tracks read, frame tracks, frame hits
    CNT_FRAME_T = 5,
    CNT_FRAME_H = 6,
    CNT_BINS_BAD = 7,         // set when the caller's bin offsets fail the check
    CNT_Q0 = 8,               // work-queue heads, one per kernel
};

__host__ __device__ inline int pstart_of(int32_t off, int b) { return ((off + 7) & ~7) + 8 * b; }

#ifdef __CUDACC__
__device__ __forceinline__ void set_status(const Work &W, int bits) { atomicOr(W.status, bits); }

// floor(a / 2^k) for signed a: arithmetic shift (two's complement, CUDA semantics)
__device__ __forceinline__ long long floor_shift(long long a, int k) { return a >> k; }
__device__ __forceinline__ long long floor_div(long long a, long long b) {
    long long q = a / b;
    if ((a % b) != 0 && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

// floor(a / b) for b > 0; operands below 2^24 in magnitude take a float quotient and an exact
// remainder correction (the quotient of the rounded division is within one of the true floor), the
// rest the 64-bit integer division.  Same result as floor_div for every input.
__device__ __forceinline__ long long floor_div_pos(long long a, long long b) {
    if (a > -(1ll << 24) && a < (1ll << 24) && b < (1ll << 24)) {
        const int ai = (int)a, bi = (int)b;
        int q = (int)floorf((float)ai / (float)bi);
        const int r = ai - q * bi;
        if (r < 0) q -= 1;
        else if (r >= bi) q += 1;
        return q;
    }
    return floor_div(a, b);
}

__device__ __forceinline__ int bin_sector(const DevGeom &g, int bin_in_event) { return bin_in_event / g.n_rows; }

// Work queue: returns the first item of the next chunk for the calling block (thread 0 grabs).
__device__ __forceinline__ int queue_next(int32_t *head, int chunk, int *sh) {
    __syncthreads();
    if (threadIdx.x == 0) *sh = atomicAdd(head, chunk);
    __syncthreads();
    return *sh;
}
#endif

// ---- launchers (host side, one per translation unit) ----------------------------------------
void launch_bins_check(const Work &W, cudaStream_t s);
void launch_grid(const Work &W, cudaStream_t s);
void launch_links(const Work &W, cudaStream_t s);
void launch_chains(const Work &W, cudaStream_t s);
void launch_follow(const Work &W, cudaStream_t s);
void launch_select(const Work &W, cudaStream_t s);
void launch_merge(const Work &W, cudaStream_t s);
void launch_frame_merge(const Work &W, cudaStream_t s);
// tracks in order of decreasing hit count into order (hist: 2 * 512 words of scratch)
void launch_len_order(const Work &W, int32_t *order, int32_t *hist, cudaStream_t s);
void launch_refit(const Work &W, const float *theta, const int32_t *order, cudaStream_t s);
// sorted: order already holds the length order of these tracks
void launch_refit_grad_fit(const Work &W, const double *theta, const float *weight, const float *anchor, int model,
                           bool grad, float *ck, long long ck_hits, long long ck_tracks, float *rec, int32_t *order,
                           int32_t *hist, bool sorted, cudaStream_t s);
void launch_refit_grad_reduce(const Work &W, double *sum_chi2, double *grad, const float *rec, double *part,
                              cudaStream_t s);
size_t refit_ck_words(long long cap_hits, long long cap_tracks);
int refit_rec_words(int cap_tracks);
int refit_part_doubles(int cap_tracks, int ns);
void launch_pack_hits(const Work &W, cudaStream_t s);
void launch_its_match(const Work &W, const float *its, int n_its, int32_t *match_trk, int32_t *match_its,
                      float *anchor, double kB, double alpha0, double dalpha, cudaStream_t s);
int its_match_nphi();
void launch_looper_pairs(const Work &W, int32_t *pair, int32_t *leg, double kB, double alpha0, double dalpha,
                         double *rec, int nt_cap, cudaStream_t s);
int loop_nphi();
int its_constants(double *out);     // 5 values
int loop_constants(double *out);    // 6 values
void prepare_kernels();
// device-wide exclusive scan of n (host) or *n_dev (device, if not NULL) int32 values; writes
// out[0..n] (out[n] = total) and *total_dev (if not NULL).
void scan_exclusive(const int32_t *in, int32_t *out, int n_cap, const int32_t *n_dev, int32_t *total_dev,
                    int32_t *tmp, int tmp_len, cudaStream_t s);
int scan_tmp_needed(int n_cap);

}  // namespace tpc
