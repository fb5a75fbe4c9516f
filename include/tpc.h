/*
 * tpc.h - C ABI of the GB300 (sm_103a) TPC track-reconstruction library.
 *
 * The library reconstructs charged-particle tracks in the 36 sectors of a time projection
 * chamber, following the tracker of arxiv 1712.09434 section 3: cellular-automaton seeding on
 * neighbouring pad rows (one thread per cluster), Kalman-filter track following and fitting (one
 * thread per track), independent sectors whose track segments are merged afterwards, and a final
 * Kalman refit.  It adds a hand-written adjoint of the refit that gives the gradient of the sum of
 * chi2 with respect to calibration parameters (the online calibration feedback of sections 2 and
 * 6), and batched tracking of many events in persistent kernels under a CUDA graph (the
 * multi-event concurrency of section 3, Table 1).
 *
 * Conventions
 *  - Every pointer in the structs below is a DEVICE pointer owned by the caller, unless stated.
 *  - Calls are stream-ordered and asynchronous on `stream` (a cudaStream_t passed as void*; NULL
 *    is the legacy default stream).  The return code covers argument validation and launch
 *    errors only.  Errors found on the device (capacity, timeout, bounds) are written to a status
 *    word in the context; tpc_sync_status() waits for the stream and returns it.
 *  - Return codes: TPC_OK (0) or a negative TPC_ERR_* value.  No call aborts or traps.
 *  - A context is not thread-safe: one host thread at a time per context.  Its calls share one
 *    workspace, so they must also be ordered on the device (the same stream, or streams joined
 *    by events); two calls of one context running concurrently on the device corrupt each other.
 *
 * Coordinates (fixed point; the reading of section 3 used by the integer decisions)
 *  - pad_fp: local y of the cluster in its sector frame in units of lsb_cm (int16).
 *  - time_fp: drift length (z_max - |z|) in units of lsb_cm (uint16, <= round(z_max/lsb_cm)).
 *  - Clusters are sorted by (event, sector, row, pad_fp, time_fp); bin_off gives the cluster range
 *    of every (event, sector, row) bin, bin = (event*n_sectors + sector)*n_rows + row.
 */
#ifndef TPC_H
#define TPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TPC_OK               0
#define TPC_ERR_INVALID_ARG  -1   /* a pointer, size or struct field is invalid              */
#define TPC_ERR_CAPACITY     -2   /* an output or workspace capacity is too small            */
#define TPC_ERR_TIMEOUT      -3   /* a bounded device-side wait or iteration limit ran out   */
#define TPC_ERR_CUDA         -4   /* a CUDA runtime call failed                              */
#define TPC_ERR_BOUNDS       -5   /* an input index or coordinate is out of range            */
#define TPC_ERR_NOT_RESERVED -6   /* the workspace is smaller than the call needs            */

#define TPC_N_TUNE 8              /* kernels with tunable launch shape                       */
#define TPC_N_PIPE_STAGES 7       /* grid, links, chains, follow, select, merge, refit        */
#define TPC_N_REFIT_STAGES 3      /* pack, refit (+adjoint), reduce                           */

/* Detector geometry (section 3; 159 pad rows at 85..247 cm, 18 sectors per side). */
typedef struct {
    int32_t n_sectors;        /* even; sectors [0, n/2) on the +z side, [n/2, n) on -z     */
    int32_t n_rows;           /* pad rows per sector, 3..512                              */
    double  x_first, x_last;  /* radii of the first and last row plane [cm], uniform pitch  */
    double  half_angle_deg;   /* half opening angle of a sector [deg]                      */
    double  z_max;            /* drift length [cm]                                         */
    double  lsb_cm;           /* fixed-point unit of pad_fp and time_fp [cm]               */
} tpc_geometry;

/* Clusters of one event (n_events = 1) or of a batch of events (concatenated, see above).
 * bin_off must run from 0 to n_clusters without decreasing.  Every call checks this on the device
 * before any kernel indexes with it; an offset set that fails is reported as TPC_ERR_BOUNDS by
 * tpc_sync_status (the call then finds no tracks and writes nothing outside its buffers). */
typedef struct {
    const int16_t  *pad_fp;   /* [n_clusters]                                              */
    const uint16_t *time_fp;  /* [n_clusters]                                              */
    const int32_t  *bin_off;  /* [n_events*n_sectors*n_rows + 1], 0 .. n_clusters, nondecr. */
    int32_t n_events;
    int32_t n_clusters;
} tpc_clusters;

/* Track output, written by tpc_track_event / tpc_track_batch (caller-owned device buffers).
 * Tracks are ordered by event, then by the index of their first segment's seed chain; hits are
 * cluster indices in track order (segments along the merge chain, ascending rows inside a
 * segment).  par = (y, z, sin phi, tan lambda, q/pT) at local x = xref in the frame of the first
 * hit's sector; cov = 15-element lower triangle, row-major; chi2 in FP32; ndf = 2*n_hits - 5, or 0
 * if the fit failed (then par, cov, chi2 are 0). */
typedef struct {
    int32_t *label;           /* [n_clusters]     track index or -1                        */
    int32_t *trk_off;         /* [cap_tracks + 1] hit range of each track                  */
    int32_t *trk_hits;        /* [cap_hits]       cluster indices                          */
    int32_t *ev_trk_off;      /* [n_events + 1]   track range of each event                */
    float   *par;             /* [cap_tracks*5]                                           */
    float   *xref;            /* [cap_tracks]                                             */
    float   *cov;             /* [cap_tracks*15]                                          */
    float   *chi2;            /* [cap_tracks]                                             */
    int32_t *ndf;             /* [cap_tracks]                                             */
    int32_t *n_tracks;        /* [1]  total number of tracks (device scalar)               */
    int32_t  cap_tracks;
    int32_t  cap_hits;
} tpc_tracks;

/* Launch shape of the tunable kernels (0 = library default).  Index: 0 grid, 1 links, 2 chains,
 * 3 follow, 4 select, 5 merge, 6 refit, 7 refit_grad.  block = threads per CTA (multiple of 32, at
 * most 256, 128, 256, 128, 1024, 512, 128, 128 by index), ctas_per_sm = CTAs per SM of the grid
 * (<= 64), chunk = work items taken per queue grab (<= 64; used by the following); for the neighbour
 * finding (index 1) chunk = 1 selects the variant that stages rows r+-1 of every bin in shared
 * memory by bulk copies (one CTA per bin) instead of reading them through L1 (one warp per bin,
 * lanes taking the bin's clusters in Z-slab order), and chunk = 2 the warp-per-bin variant whose
 * lanes take the clusters in cluster (Y, Z) order; for the gradient kernel (index 7) the default
 * recomputes the Kalman states of the reverse sweep from checkpoints every 16 steps, and chunk = 1
 * selects the variant that stores the input state of every step instead (80 B per hit of
 * workspace, no recomputation; the same gradient bit for bit).
 * Launch shapes never change results. */
typedef struct {
    int32_t block[TPC_N_TUNE];
    int32_t ctas_per_sm[TPC_N_TUNE];
    int32_t chunk[TPC_N_TUNE];
} tpc_tuning;

typedef struct tpc_ctx tpc_ctx;

/* Create a context on the current CUDA device.  Bz in tesla.  Geometry tables are derived on the
 * host and uploaded.  *out receives the context.  Errors: INVALID_ARG, CUDA. */
int tpc_init(const tpc_geometry *geom, double bz_tesla, tpc_ctx **out);

/* Size the library-owned workspace for calls of up to max_clusters clusters and max_events
 * events (grows, never shrinks; allocation happens only here and in tpc_init).  Any call whose
 * size exceeds the reservation fails with TPC_ERR_NOT_RESERVED.  Errors: INVALID_ARG, CUDA. */
int tpc_reserve(tpc_ctx *ctx, int32_t max_clusters, int32_t max_events);

/* Release the context and its workspace.  NULL is ignored. */
void tpc_destroy(tpc_ctx *ctx);

/* Track one or more events with one launch per step (the plain, per-event form; no graph).
 * Steps: grid, neighbour finding, link cleaning and chains, following, selection, merge, refit at
 * the nominal calibration.  `in` and `out` as documented above.  Errors: INVALID_ARG,
 * NOT_RESERVED, CUDA; device-side errors via tpc_sync_status. */
int tpc_track_event(tpc_ctx *ctx, const tpc_clusters *in, tpc_tracks *out, void *stream);

/* Same result as tpc_track_event (bit-identical hit assignment), for a batch of events: the same
 * persistent work-queue kernels, captured once into a CUDA graph and replayed.  The graph is keyed
 * by the complete argument set (buffers, sizes, tuning); a call with different arguments captures
 * again and updates the executable graph in place.  tune may be NULL (library defaults). */
int tpc_track_batch(tpc_ctx *ctx, const tpc_clusters *in, tpc_tracks *out, const tpc_tuning *tune,
                    void *stream);

/* Kalman refit of the tracks in `trk` (trk_off, trk_hits and n_tracks as written by a tracking
 * call on the same clusters; the other output pointers are not used) with clusters transformed
 * under calibration theta = [s_vd, d_0..d_{ns-1}, a_0..a_{ns-1}] (1 + 2*n_sectors doubles, device).
 * Transform: z = side*(z_max - s_vd*D) + d_k and (x, y) = (x_r, y)*(1 + a_k*(rho - x_first)/
 * ((x_last - x_first)*rho)), rho = |(x_r, y)|.  Objective: sum over fitted tracks of
 * weight[t]*chi2[t] (weight: device float [n_tracks], or NULL for all 1; a track of weight 0 is
 * skipped), written to *sum_chi2 (device double); if grad is not NULL, its gradient
 * d(objective)/d(theta) (device, 1 + 2*n_sectors doubles) from the adjoint of the refit.  FP32
 * Kalman arithmetic; FP64 cross-track reductions in a fixed order (deterministic).
 * anchor (device float [n_tracks][8], 16-byte aligned, or NULL): reference measurements at the
 * production vertex that make the calibration identifiable (section 6: drift calibration against
 * inner-tracker tracks).  Per track: [0] sigma_v of the vertex point (y, z) = (0, 0) at x = 0 in
 * the frame of the first hit's sector; [1], [2] z0 and its sigma; [3], [4] tan lambda and sigma;
 * [5], [6] q/pT and sigma; [7] unused.  A sigma <= 0 leaves its term out; a track with any term
 * takes the exact helix step from its first hit to x = 0 (a failed step drops the track) and adds
 * the chi2 of each term to chi2[t].
 * error_model: TPC_ERRORS_FIXED takes measurement errors sigma = 0.1 cm in the calibrated y and z
 * (the fit of the tracking); TPC_ERRORS_RAW takes them in the raw coordinates and carries them
 * through the transformation (sigma (1 + a_k g) in y, sigma s_vd in z, g the radial factor above),
 * which makes the objective -2 log L up to a constant for Gaussian raw errors: with fixed
 * calibrated errors a theta that shrinks the data also shrinks the residuals, and the minimum of
 * the sum of chi2 is biased towards it.
 * Errors: INVALID_ARG (also a misaligned anchor or an unknown error_model), NOT_RESERVED, CUDA;
 * device-side errors via tpc_sync_status. */
#define TPC_ERRORS_FIXED 0
#define TPC_ERRORS_RAW 1
int tpc_refit_grad(tpc_ctx *ctx, const tpc_clusters *in, const tpc_tracks *trk, const double *theta,
                   const float *weight, const float *anchor, int32_t error_model, double *sum_chi2, double *grad,
                   void *stream);

/* One whole step as a single CUDA graph launch: the tracking of tpc_track_batch (S1-S8) followed by
 * tpc_refit_grad (S0, S8, S9) on the tracks just found, captured together once per argument set and
 * replayed (a call with other arguments captures again).  Arguments as for the two calls; the
 * refit reads the track count from out->n_tracks on the device.  Results are bit-identical to the
 * two calls made one after the other.  Errors: as tpc_track_batch and tpc_refit_grad. */
int tpc_track_refit_batch(tpc_ctx *ctx, const tpc_clusters *in, tpc_tracks *out, const double *theta,
                          const float *weight, const float *anchor, int32_t error_model, double *sum_chi2,
                          double *grad, const tpc_tuning *tune, void *stream);

/* TPC-ITS matching for the drift calibration (sections 2.1 and 6 of the paper: the TPC drift is
 * calibrated by matching TPC tracks to tracks of the inner tracker, ITS).
 *  - in: the clusters the tracks were found on; trk: tracks with their fit (trk_off, trk_hits, par,
 *    cov, xref, ndf, n_tracks as a tracking call writes them).
 *  - its: device float [n_its][8] = (phi0, z0, tan lambda, q/pT, sigma_phi0, sigma_z0, sigma_tl,
 *    sigma_qpt): global azimuth of the momentum, z and direction at the production vertex, and their
 *    errors.  n_its <= the context's chain capacity (clusters / 5), else TPC_ERR_CAPACITY.
 *  - Rule: every fitted track is carried by the exact helix step (FP64) from its first hit to
 *    x = 0 in the frame of that hit's sector k; an ITS track is taken in that frame as y = 0,
 *    sin phi = sin(phi0 - alpha_k).  Candidates lie within 0.1 rad in azimuth, 0.1 in tan lambda and
 *    2 cm in z (z is what the calibration corrects); chi2 over (y, sin phi, tan lambda, q/pT) with the
 *    track's covariance plus (0.01 cm)^2 in y and the ITS errors, chi2 <= 100 (loose: before the
 *    calibration the track parameters carry the distortion, and a tight gate would pick references
 *    by their own noise).  Mutual best pairs by (floor(chi2 * 2^20), index) are matched.
 *  - Outputs (device): match_trk [n_tracks] (ITS index or -1), match_its [n_its] (track or -1), and
 *    if anchor is not NULL (float [n_tracks][8], 16-byte aligned) the reference measurements of
 *    tpc_refit_grad for every matched track that starts within the first 8 pad rows, has at least
 *    30 hits and |sin phi| < 0.9 at the vertex: (0.01, z0, sigma_z0, tan lambda, sigma_tl, q/pT,
 *    sigma_qpt, 0); zeros for the others.
 * Errors: INVALID_ARG, NOT_RESERVED, CAPACITY, CUDA; BOUNDS (a hit outside the clusters) via
 * tpc_sync_status. */
int tpc_its_match(tpc_ctx *ctx, const tpc_clusters *in, const tpc_tracks *trk, const float *its, int32_t n_its,
                  int32_t *match_trk, int32_t *match_its, float *anchor, void *stream);

/* Looper-leg pairing (section 3 of the paper merges the track segments that the sector tracking
 * finds; this joins the two legs of a low-pT looper, which leave the tracking as two tracks).
 *  - in: the clusters the tracks were found on; trk: tracks with their fit (trk_off, trk_hits, par,
 *    xref, ndf, n_tracks as a tracking call writes them).  Tracks beyond the context's chain
 *    capacity (clusters / 5) are not considered (TPC_ERR_CAPACITY via tpc_sync_status).
 *  - Rule: both legs are fitted outwards in pad-row order, so the returning leg has the opposite
 *    curvature and tan lambda of the outgoing one on the same circle.  From every fitted state (at
 *    the first hit, in that hit's sector frame; FP64): the centre of curvature in the global frame,
 *    the radius R = 1/|C| and the z reached at the point of the circle farthest from the beam, along
 *    the fitted direction.  Candidates have R <= 130 cm and a centre >= 40 cm from the beam.  Two
 *    candidates of one event with opposite curvature pair if their centres are within 5 cm, radii
 *    within 5 cm, far-point z within 8 cm and |tan lambda_a + tan lambda_b| <= 0.05; mutual best
 *    pairs by (floor(D * 2^20), index), D = dcentre^2 + dR^2 + dz^2 (cm^2), are joined.
 *  - Outputs (device, [n_tracks]): pair[t] = the other leg or -1; if leg is not NULL, leg[t] = 1 for
 *    the outgoing leg (the one whose |z| grows outwards; the lower index if both tan lambda are
 *    equal), 2 for the returning leg, 0 for an unpaired track.  The joined looper is the outgoing
 *    leg's hits followed by the returning leg's in reverse order; each leg keeps its own fit.
 * Errors: INVALID_ARG, NOT_RESERVED, CAPACITY, CUDA; BOUNDS (a hit outside the clusters) via
 * tpc_sync_status. */
int tpc_looper_pairs(tpc_ctx *ctx, const tpc_clusters *in, const tpc_tracks *trk, int32_t *pair, int32_t *leg,
                     void *stream);

/* Time-frame slice merge (arxiv 1712.09434 section 3, its outlook for continuous readout: a time
 * frame of many overlapping collisions is cut along the drift-time axis, the slices are tracked
 * one by one, and the track segments are merged afterwards).
 *  - in: the clusters of n_events = n_slices consecutive slices of slice_len LSB of readout time,
 *    in the batch layout (bin = (slice*n_sectors + sector)*n_rows + row) with slice-local times:
 *    a cluster read out at time tau lies in slice floor(tau / slice_len) with time_fp = tau -
 *    slice*slice_len < slice_len (a track starting at a later time is a BOUNDS error).
 *    1 <= slice_len <= round(z_max/lsb_cm) + 1.
 *  - slice_trk: the tracks of every slice as tpc_track_batch writes them for `in` (trk_off,
 *    trk_hits, ev_trk_off and n_tracks are read; device).  At most the context's chain capacity.
 *  - frame (outputs, device): label [n_clusters] (frame track id or -1), trk_off [cap_tracks + 1],
 *    trk_hits [cap_hits] (cluster indices; the hits of the chain's slice tracks, in chain order),
 *    n_tracks [1], and ev_trk_off [2] = {0, n_tracks} if not NULL.  The other pointers are not
 *    used and may be NULL.
 * Rule: readout time falls outwards along a track, so the piece of a track in slice j+1 ends, at
 * its outer end, where its piece in slice j begins.  The outer end of a slice-(j+1) track (its last
 * hit and the hit 3 positions earlier, on (round(x_row/lsb), pad_fp, time_fp + slice_len)) is
 * rotated into the frame of the first hit of a slice-j track when that lies in an adjacent sector
 * of the same side (round(cos, sin 20 deg * 2^30), floor shifts), extrapolated linearly (floor
 * division) to that track's first row (at most 2048 LSB away) and compared with the merge windows
 * |dY|, |dZ| <= 192; D = dY^2 + dZ^2.  Mutual best pairs by (D, track index) are linked; a chain of
 * links is one frame track, ordered by the index of its first slice track.  The links of the last
 * call are what tpc_debug_copy 9 returns.
 * Errors: INVALID_ARG, NOT_RESERVED, CUDA; device-side errors (CAPACITY: more slice tracks than the
 * chain capacity, or more frame tracks or hits than cap_tracks / cap_hits; BOUNDS: a track offset
 * or hit outside the clusters) via tpc_sync_status. */
int tpc_merge_slices(tpc_ctx *ctx, const tpc_clusters *in, const tpc_tracks *slice_trk, int32_t slice_len,
                     tpc_tracks *frame, void *stream);

/* Set the launch shapes that later calls of this context use when they pass none (tpc_track_event,
 * tpc_refit_grad, and tpc_track_batch with tune == NULL); NULL restores the library defaults.
 * The values are copied.  Errors: INVALID_ARG (a value outside the bounds of tpc_tuning). */
int tpc_set_tuning(tpc_ctx *ctx, const tpc_tuning *tune);

/* Optional rules for data with missing clusters (dead pad rows, cluster inefficiency): readings of
 * the paper's CA on neighbouring pad rows and of its segment merging (section 3).  Bits:
 *  - TPC_RULE_SKIP_ROW: a cluster whose neighbouring row r+1 (r-1) has no cluster inside the link
 *    window |dY|, |dZ| <= 384 looks at row r+2 (r-2) with the window doubled; with the partners a and
 *    b rows away the straight-line residual is e = b Yu + a Yd - (a+b) Yc (likewise in Z), the cut
 *    6 (ey^2 + ez^2) <= (a^2 + b^2 + (a+b)^2) * 13600, the pair of minimum (D, u, d) wins.  Chains
 *    may then skip a row; the following's filter steps once per row across it.
 *  - TPC_RULE_GAP_MERGE: two accepted segments of one sector whose ends are k = 9..GAP_MAX rows apart
 *    (at least 8 empty rows, which the following does not bridge) are joined when the integer filter
 *    of each, run over its kept hits and extrapolated row by row across the gap under the
 *    following's stop rules, meets the other's end within the following's radius after k - 1
 *    misses (77 + 38 (k - 1) LSB); D is the sum of both squared distances, mutual best pairs by
 *    (D, index).  For the sector merge a segment with a gap successor is no outer end and one with
 *    a gap predecessor no first segment.
 * 0 (the default) gives the plain readings.  The rules apply to later tracking calls of the context.
 * Errors: INVALID_ARG (unknown bits). */
#define TPC_RULE_SKIP_ROW  1
#define TPC_RULE_GAP_MERGE 2
int tpc_set_rules(tpc_ctx *ctx, int32_t rules);

/* The rule bits and GAP_MAX, for comparison with an independent implementation.  Returns the count
 * written (at most cap). */
int tpc_rule_constants(int64_t *out, int32_t cap);

/* The reading constants of the matching steps, for comparison with an independent implementation:
 * TPC-ITS matching (sigma_y of an ITS track at the vertex, azimuth window, tan lambda window, z window,
 * chi2 gate), then looper-leg pairing (largest radius, smallest centre distance from the beam,
 * centre, radius and far-point z gates in cm, tan lambda sum gate).  Writes min(n, cap) values to out
 * (host) and returns n = 11. */
int tpc_match_constants(double *out, int32_t cap);

/* Wait for `stream` and return the device status word of the last calls (then clear it). */
int tpc_sync_status(tpc_ctx *ctx, void *stream);

/* Static description of a return code. */
const char *tpc_strerror(int code);

/* Copy an internal intermediate of the last tracking call to `dst` (device, caller-owned) for
 * step-by-step parity tests (int32 arrays; N = reserved clusters, C = chain capacity):
 * 0 up[N], 1 down[N] (neighbour links, -1 = none), 2 n_chains[1], 3 chain_start[C],
 * 4 chain_len[C], 5 cand_n[C], 6 cand_slots[C*n_rows] (cluster per row, -1 = miss, valid inside
 * the candidate's row range), 7 cand_rows[C] (first row | last row << 16), 8 seg_n[C] (kept hits,
 * 0 if rejected), 9 next[C] (merge successor or -1; after tpc_merge_slices, the successor of every slice
 * track in the next-earlier slice), 10 counters[16] (0 chains, 1 tracks, 2 hits,
 * 3 largest number of selection rounds), 11 the per-track records of the last tpc_refit_grad
 * (26 floats per track: weighted chi2, d/ds_vd, then 8 x (sector as int32 bits or -1, d/dd_k,
 * d/da_k); a track that was not fitted has chi2 0).  At most dst_bytes bytes are copied. */
int tpc_debug_copy(tpc_ctx *ctx, int32_t what, void *dst, int64_t dst_bytes, void *stream);

/* Per-stage timing.  tpc_profile_enable(ctx, 1) makes later calls record CUDA events between their
 * stages on the call's stream (inside the CUDA graph for tpc_track_batch).  tpc_profile_read waits
 * for the last profiled calls, adds their stage times to per-context sums and copies the sums
 * (milliseconds) to ms[0..cap): the TPC_N_PIPE_STAGES tracking stages, then the
 * TPC_N_REFIT_STAGES refit stages; *n_calls (may be NULL) receives the number of tracking calls
 * summed.  Only the last call of each kind since the previous read is counted, so read after every
 * call.  A negative cap resets the sums (nothing is copied).  Returns the number of stages. */
int tpc_profile_enable(tpc_ctx *ctx, int enable);
int tpc_profile_read(tpc_ctx *ctx, double *ms, int32_t cap, int32_t *n_calls);

/* Neighbour finding for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a library convenience.  Callers recording work into a CUDA graph by stream
 * capture (cudaMalloc cannot be captured), plug-ins whose host framework owns all GPU memory, and
 * real-time code that may only allocate at start-up can compute the neighbour links of
 * tpc_track_event (the same kernels; up/down as returned by tpc_debug_copy 0 and 1) without a
 * context or a workspace.  The scratch lives in a static device array of the library, which
 * every GPU that loads the library keeps until the process exits (about 9 MB): it limits a call
 * to TPC_NOALLOC_MAX_CLUSTERS clusters and TPC_NOALLOC_MAX_BINS (event, sector, row) bins; larger
 * inputs return TPC_ERR_CAPACITY with a message on stderr.  The call allocates nothing.
 *  - geom: host struct (only n_sectors and n_rows are used); in: device clusters as for
 *    tpc_track_event; up, down: device int32 [n_clusters] outputs (-1 = no link); status: device
 *    int32 [1] receiving the device-side status bits (0 = ok; may be NULL).
 *  - The first call on a device looks up the array's device address and sets a kernel attribute;
 *    make that first call outside any stream capture.  Later calls only enqueue work on `stream`.
 *  - All calls on a device share the array: calls that overlap on the GPU (different streams,
 *    or graph launches running concurrently) race and corrupt each other's results.  The array
 *    keeps the last call's contents; the call clears what must start at zero.
 *  - The device address found by the first call is kept for the life of the process.  A process
 *    that resets a device (cudaDeviceReset) gets a new copy of the array at another address and
 *    must not call this entry point on that device again.
 *  - bin_off is checked as for tpc_track_event: an offset set that does not run from 0 to
 *    n_clusters without decreasing sets TPC_ERR_BOUNDS in *status and no link is made.
 * Errors: INVALID_ARG, CAPACITY, CUDA. */
#define TPC_NOALLOC_MAX_CLUSTERS (1 << 20)
#define TPC_NOALLOC_MAX_BINS 16384
int tpc_links_noalloc(const tpc_geometry *geom, const tpc_clusters *in, int32_t *up, int32_t *down,
                      int32_t *status, void *stream);

/* Self-test of the failure path of a bounded device-side wait: a kernel waits on an mbarrier that
 * nothing arrives at, gives up after spin_limit (1..2^20) polls, writes TPC_ERR_TIMEOUT to *status
 * (device int32) and returns; the context stays usable.  The paper has no counterpart
 * (diagnostics).
 * Errors: INVALID_ARG, CUDA. */
int tpc_selftest_wait_timeout(int32_t *status, int32_t spin_limit, void *stream);

/* FP32 fused multiply-add throughput (diagnostic; the paper has no counterpart): the roof of the
 * Kalman refit and its adjoint, which are FP32 arithmetic per thread.  Launches sms * ctas_per_sm
 * CTAs of `threads` threads (multiple of 32, <= 256) that each run 8 independent FMA chains for
 * iters * 16 steps and store one float each to out (device, [sms * ctas_per_sm * threads]);
 * *flops (host) receives the floating-point operations of the launch (an FMA counts two).  Time
 * it with events on `stream`.  Errors: INVALID_ARG, CUDA. */
int tpc_fma_peak(float *out, int64_t iters, int32_t ctas_per_sm, int32_t threads, int64_t *flops, void *stream);

/* Reading constants of the integer track finding, for comparison with an independent
 * implementation: W_LINK, D_MAX, N_SEED, M_MISS, W_F0, W_F1, V_MAX, N_MIN, W_MERGE, MERGE_XMAX,
 * MERGE_BACK.  Returns the count written (at most cap). */
int tpc_constants(int64_t *out, int32_t cap);

#ifdef __cplusplus
}
#endif

#endif /* TPC_H */
