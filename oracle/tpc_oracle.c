/*
 * Plain CPU oracle for the TPC track reconstruction hot path (test infrastructure only).
 *
 * This file is the slow, obviously-correct reference that the CUDA path is checked against.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant generator with the CUDA library: every constant
 * below is declared here on its own, and a test compares the two sets of values.
 *
 * Steps follow the paper's tracker (section 3): cellular-automaton seeding on neighbouring pad
 * rows (neighbour finding, link cleaning, seed chains of five to ten hits), Kalman-filter
 * track following and fitting, independent sectors whose segments are merged afterwards, and a
 * final track refit.  The paper fixes only this structure; every constant, rounding rule and
 * tie-break is a stated reading (listed in the design notes) and is written out here in plain
 * loops.  Integer decisions use int64; the fit uses double precision throughout.
 *
 * Parity status: links (brute force), selection (naive greedy), the partition invariant, the fit
 * (noise-free helices, chi2 statistics, least-squares optimum) and the gradient (central
 * differences of this file's own objective) are pinned by the CPU tests; the time-frame slice
 * merge by a constructed track cut by a slice boundary, the single-slice and whole-slice-delay
 * invariances and the truth of its links; the rules for inefficient data, the TPC-ITS matching
 * and the looper-leg pairing by constructed cases at every window edge, exact tracks and the truth
 * of their decisions on generated events.  Track-finding efficiency on these synthetic events
 * has no printed value in the paper: parity unpinned.
 */
#define _USE_MATH_DEFINES
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- reading constants (integer track finding, LSB = 1/128 cm) ---------------------------- */
#define OR_W_LINK      384      /* neighbour window in Y and Z, |dY|,|dZ| <= 3 cm             */
#define OR_D_MAX       13600    /* max squared second difference of a link triplet (LSB^2)    */
#define OR_N_SEED      5        /* minimum chain length kept as a seed                        */
#define OR_M_MISS      8        /* following stops after this many consecutive empty rows     */
#define OR_W_F0        77       /* following search radius, no miss (LSB)                     */
#define OR_W_F1        38       /* growth of the radius per consecutive miss (LSB)            */
#define OR_V_MAX       320      /* following stops when |dY/row| exceeds this (LSB per row)   */
#define OR_N_MIN       10       /* minimum kept hits of an accepted track segment             */
#define OR_W_MERGE     192      /* merge window in Y and Z (LSB)                              */
#define OR_MERGE_XMAX  2048     /* maximum merge extrapolation distance (LSB)                 */
#define OR_MERGE_BACK  3        /* direction baseline of a segment end, in hits               */
#define OR_MAX_ROWS    512

/* ---- optional rules for inefficient data (readings of the paper's CA on neighbouring rows and
 *      of its segment merging; off by default) ------------------------------------------------ */
#define OR_RULE_SKIP_ROW  1     /* a link may skip one row where row r+-1 has no candidate      */
#define OR_RULE_GAP_MERGE 2     /* segments of one sector are joined across a gap of rows       */
#define OR_GAP_MAX        24    /* largest row distance between the two ends of a gap link      */

/* ---- reading constants (fit) ------------------------------------------------------------- */
#define OR_SIGMA2      0.01     /* measurement variance of y and z (cm^2)                     */
#define OR_SNP_MAX     0.999    /* |sin phi| limit of the local helix parametrisation          */
#define OR_CPHI_MIN    0.01     /* minimum cos phi after a sector rotation                    */
#define OR_CLIGHT      0.299792458e-2
#define OR_PI          3.14159265358979323846

typedef struct {
    int32_t n_sectors, n_rows;
    double x_first, x_last, half_angle_deg, z_max, lsb, bz;
} or_geom_in;

typedef struct {
    int n_sectors, n_rows;
    double lsb, z_max, kB, half_angle;
    double xr[OR_MAX_ROWS];
    int64_t ymax[OR_MAX_ROWS];  /* floor(x_r tan(half angle) / lsb)   */
    int64_t xtab[OR_MAX_ROWS];  /* round(x_r / lsb)                   */
    int64_t zmax;               /* round(z_max / lsb)                 */
    int64_t c30, s30;           /* round(cos, sin(2*half angle) 2^30) */
} or_geom;

static int64_t round_half_away(double v) { return (int64_t)(v < 0 ? -floor(-v + 0.5) : floor(v + 0.5)); }

static int make_geom(const or_geom_in *in, or_geom *g) {
    if (!in || in->n_rows < 3 || in->n_rows > OR_MAX_ROWS || in->n_sectors < 1) return -1;
    g->n_sectors = in->n_sectors;
    g->n_rows = in->n_rows;
    g->lsb = in->lsb;
    g->z_max = in->z_max;
    g->kB = -OR_CLIGHT * in->bz;
    g->half_angle = in->half_angle_deg * OR_PI / 180.0;
    for (int r = 0; r < in->n_rows; r++) {
        double x = in->x_first + r * (in->x_last - in->x_first) / (in->n_rows - 1);
        g->xr[r] = x;
        g->ymax[r] = (int64_t)floor(x * tan(g->half_angle) / in->lsb);
        g->xtab[r] = round_half_away(x / in->lsb);
    }
    g->zmax = round_half_away(in->z_max / in->lsb);
    g->c30 = round_half_away(cos(2.0 * g->half_angle) * 1073741824.0);
    g->s30 = round_half_away(sin(2.0 * g->half_angle) * 1073741824.0);
    return 0;
}

/* floor(a / 2^k) and floor(a / b), written out so that no signed-shift convention is assumed. */
static int64_t floor_shift(int64_t a, int k) {
    int64_t d = (int64_t)1 << k;
    int64_t q = a / d;
    if ((a % d) != 0 && a < 0) q -= 1;
    return q;
}
static int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b) != 0 && ((a < 0) != (b < 0))) q -= 1;
    return q;
}
static int64_t iabs64(int64_t a) { return a < 0 ? -a : a; }

/* Bin (sector*n_rows + row) of every cluster, from the per-bin offsets. */
static int32_t *cluster_bins(const int32_t *bin_off, int nbins, int32_t n) {
    int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (int k = 0; k < nbins; k++)
        for (int32_t c = bin_off[k]; c < bin_off[k + 1]; c++) b[c] = k;
    return b;
}

/* First index in [lo, hi) of a pad-sorted bin with pad >= y. */
static int32_t lower_pad(const int16_t *pad, int32_t lo, int32_t hi, int64_t y) {
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if ((int64_t)pad[mid] < y) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* ============================================================================================
 * S2  Neighbour finding (cellular automaton, one decision per cluster; section 3).
 * For cluster c on row r (1 <= r <= n_rows-2) choose, among clusters u on row r+1 and d on row
 * r-1 of the same sector that lie within the window |dY|, |dZ| <= W_LINK of c, the pair with the
 * smallest squared second difference D = (Yu+Yd-2Yc)^2 + (Zu+Zd-2Zc)^2 <= D_MAX; ties go to the
 * smaller (u, d).  The candidates are enumerated by scanning the pad-sorted bin; no grid.
 *
 * With OR_RULE_SKIP_ROW a side whose neighbouring row has no cluster inside the window looks one
 * row further (rows r+-2) with the window doubled.  With the up partner a rows and the down
 * partner b rows away, the straight-line residual is e = b Yu + a Yd - (a+b) Yc (and likewise in
 * Z); its variance is k = a^2 + b^2 + (a+b)^2 times that of one coordinate, so the cut becomes
 * 6 D <= k D_MAX (for a = b = 1 the rule above).  a and b are fixed per cluster, so the pairs of
 * one cluster are still ranked by D.
 * ========================================================================================== */
static int window_list(const int16_t *pad, const uint16_t *tim, const int32_t *bin_off, int b, int64_t yc,
                       int64_t zc, int64_t w, int32_t *list) {
    int m = 0;
    for (int32_t u = lower_pad(pad, bin_off[b], bin_off[b + 1], yc - w); u < bin_off[b + 1] && pad[u] <= yc + w; u++)
        if (iabs64((int64_t)tim[u] - zc) <= w) list[m++] = u;
    return m;
}

int or_links_rules(const or_geom_in *gin, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off,
                   int32_t n, int32_t rules, int32_t *up, int32_t *down) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    for (int32_t c = 0; c < n; c++) { up[c] = -1; down[c] = -1; }
    int32_t *ulist = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
    int32_t *dlist = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
    const int skip = (rules & OR_RULE_SKIP_ROW) != 0;
    for (int s = 0; s < g.n_sectors; s++) {
        for (int r = 1; r < g.n_rows - 1; r++) {
            int b = s * g.n_rows + r;
            for (int32_t c = bin_off[b]; c < bin_off[b + 1]; c++) {
                int64_t yc = pad[c], zc = tim[c];
                int64_t a = 1, bd_ = 1;
                int nu = window_list(pad, tim, bin_off, b + 1, yc, zc, OR_W_LINK, ulist);
                if (nu == 0 && skip && r + 2 <= g.n_rows - 1) {
                    nu = window_list(pad, tim, bin_off, b + 2, yc, zc, 2 * OR_W_LINK, ulist);
                    a = 2;
                }
                int nd = window_list(pad, tim, bin_off, b - 1, yc, zc, OR_W_LINK, dlist);
                if (nd == 0 && skip && r - 2 >= 0) {
                    nd = window_list(pad, tim, bin_off, b - 2, yc, zc, 2 * OR_W_LINK, dlist);
                    bd_ = 2;
                }
                const int64_t k = a * a + bd_ * bd_ + (a + bd_) * (a + bd_);
                int64_t bestD = -1;
                int32_t bu = -1, bd = -1;
                for (int i = 0; i < nu; i++) {
                    for (int j = 0; j < nd; j++) {
                        int32_t u = ulist[i], d = dlist[j];
                        int64_t ey = bd_ * (int64_t)pad[u] + a * (int64_t)pad[d] - (a + bd_) * yc;
                        int64_t ez = bd_ * (int64_t)tim[u] + a * (int64_t)tim[d] - (a + bd_) * zc;
                        int64_t D = ey * ey + ez * ez;
                        if (6 * D > k * OR_D_MAX) continue;
                        if (bestD < 0 || D < bestD || (D == bestD && (u < bu || (u == bu && d < bd)))) {
                            bestD = D; bu = u; bd = d;
                        }
                    }
                }
                up[c] = bu;
                down[c] = bd;
            }
        }
    }
    free(ulist);
    free(dlist);
    return 0;
}

int or_links(const or_geom_in *gin, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off,
             int32_t n, int32_t *up, int32_t *down) {
    return or_links_rules(gin, pad, tim, bin_off, n, 0, up, down);
}

/* S3  Link cleaning: keep a link only when it is mutual (both sides read the uncleaned links). */
int or_clean(int32_t n, const int32_t *up, const int32_t *down, int32_t *up2, int32_t *down2) {
    for (int32_t c = 0; c < n; c++) {
        up2[c] = (up[c] >= 0 && down[up[c]] == c) ? up[c] : -1;
        down2[c] = (down[c] >= 0 && up[down[c]] == c) ? down[c] : -1;
    }
    return 0;
}

/* S4  Chains: a start has an outgoing but no incoming cleaned link; follow up-links to the end.
 * Chains of at least N_SEED hits are kept, ordered by start cluster.  Returns the count, or -2 if
 * cap is too small. */
int32_t or_chains(int32_t n, const int32_t *up2, const int32_t *down2, int32_t *chain_start,
                  int32_t *chain_len, int32_t cap) {
    int32_t nc = 0;
    for (int32_t c = 0; c < n; c++) {
        if (up2[c] < 0 || down2[c] >= 0) continue;
        int32_t len = 0;
        for (int32_t x = c; x >= 0; x = up2[x]) len++;
        if (len < OR_N_SEED) continue;
        if (nc >= cap) return -2;
        chain_start[nc] = c;
        chain_len[nc] = len;
        nc++;
    }
    return nc;
}

/* ---- S5 helpers: integer steady-state Kalman filter (alpha-beta-gamma, Q16 fixed point) ---- */
typedef struct { int64_t p, v, a; } abg;

/* State at m0 with the velocity of the step to m1, drow >= 1 rows further: floor((m1 - m0) 2^16 /
 * drow) per row (exact for drow = 1 or 2, a row skipped by a link). */
static void abg_init(abg *f, int64_t m0, int64_t m1, int64_t drow) {
    f->p = m0 * 65536; f->v = floor_div((m1 - m0) * 65536, drow); f->a = 0;
}
static void abg_predict(abg *f) { f->p += f->v + floor_shift(f->a, 1); f->v += f->a; }
static void abg_update(abg *f, int64_t m) {
    int64_t e = m * 65536 - f->p;
    f->p += floor_shift(e, 1);   /* alpha = 1/2  */
    f->v += floor_shift(e, 3);   /* beta  = 1/8  */
    f->a += floor_shift(e, 5);   /* gamma = 1/32 */
}
static int64_t q16_round(int64_t p) { return floor_shift(p + 32768, 16); }

/* Nearest cluster of bin b to (py, pz) within radius w: minimum (d^2, index), or -1. */
static int32_t nearest(const int16_t *pad, const uint16_t *tim, const int32_t *bin_off, int b,
                       int64_t py, int64_t pz, int64_t w) {
    int64_t best = -1;
    int32_t bx = -1;
    for (int32_t x = lower_pad(pad, bin_off[b], bin_off[b + 1], py - w); x < bin_off[b + 1] && pad[x] <= py + w; x++) {
        int64_t dy = pad[x] - py, dz = tim[x] - pz;
        int64_t d2 = dy * dy + dz * dz;
        if (d2 > w * w) continue;
        if (best < 0 || d2 < best) { best = d2; bx = x; }
    }
    return bx;
}

/* Extend one direction: `hits` is the chain in filter order (first element farthest from the
 * extension side), rows[] their pad rows.  The filter steps once per pad row: a row that the chain
 * skips (a link across an empty row) is a prediction without an update.  Appends found clusters
 * to out[] in the order they are found. */
static int follow_dir(const or_geom *g, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off,
                      int sector, const int32_t *hits, const int *rows, int nh, int row_last, int dir,
                      int32_t *out) {
    abg fy, fz;
    int64_t d01 = iabs64(rows[1] - rows[0]);
    abg_init(&fy, pad[hits[0]], pad[hits[1]], d01);
    abg_init(&fz, tim[hits[0]], tim[hits[1]], d01);
    for (int k = 1; k < nh; k++) {
        for (int64_t j = iabs64(rows[k] - rows[k - 1]); j > 0; j--) { abg_predict(&fy); abg_predict(&fz); }
        abg_update(&fy, pad[hits[k]]); abg_update(&fz, tim[hits[k]]);
    }
    int nout = 0, misses = 0;
    for (int row = row_last + dir; row >= 0 && row < g->n_rows; row += dir) {
        abg_predict(&fy); abg_predict(&fz);
        int64_t py = q16_round(fy.p), pz = q16_round(fz.p);
        if (iabs64(py) > g->ymax[row] || pz < 0 || pz > g->zmax || iabs64(fy.v) > (int64_t)OR_V_MAX * 65536) break;
        int64_t w = OR_W_F0 + (int64_t)OR_W_F1 * misses;
        int32_t x = nearest(pad, tim, bin_off, sector * g->n_rows + row, py, pz, w);
        if (x >= 0) {
            abg_update(&fy, pad[x]); abg_update(&fz, tim[x]);
            out[nout++] = x;
            misses = 0;
        } else if (++misses >= OR_M_MISS) {
            break;
        }
    }
    return nout;
}

/* S5  Track following (section 3: Kalman filter track following over the pad rows).
 * Each chain is extended inwards and outwards row by row; candidate hit lists are written in
 * ascending row order, n_rows slots per candidate. */
int or_follow(const or_geom_in *gin, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off,
              int32_t n, int32_t n_chains, const int32_t *chain_start, const int32_t *chain_len,
              const int32_t *up2, int32_t *cand_hits, int32_t *cand_n) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    int nbins = g.n_sectors * g.n_rows;
    int32_t *bins = cluster_bins(bin_off, nbins, n);
    int32_t chain[OR_MAX_ROWS], rev[OR_MAX_ROWS], ext_in[OR_MAX_ROWS], ext_out[OR_MAX_ROWS];
    int crow[OR_MAX_ROWS], rrow[OR_MAX_ROWS];
    for (int32_t t = 0; t < n_chains; t++) {
        int nh = 0;
        for (int32_t x = chain_start[t]; x >= 0 && nh < OR_MAX_ROWS; x = up2[x]) chain[nh++] = x;
        if (nh != chain_len[t]) { free(bins); return -3; }
        int sector = bins[chain[0]] / g.n_rows;
        for (int k = 0; k < nh; k++) crow[k] = bins[chain[k]] % g.n_rows;
        int r_first = crow[0], r_last = crow[nh - 1];
        int n_out = follow_dir(&g, pad, tim, bin_off, sector, chain, crow, nh, r_last, +1, ext_out);
        for (int k = 0; k < nh; k++) { rev[k] = chain[nh - 1 - k]; rrow[k] = crow[nh - 1 - k]; }
        int n_in = follow_dir(&g, pad, tim, bin_off, sector, rev, rrow, nh, r_first, -1, ext_in);
        int32_t *o = cand_hits + (int64_t)t * g.n_rows;
        int m = 0;
        for (int k = n_in - 1; k >= 0; k--) o[m++] = ext_in[k];
        for (int k = 0; k < nh; k++) o[m++] = chain[k];
        for (int k = 0; k < n_out; k++) o[m++] = ext_out[k];
        cand_n[t] = m;
        for (int k = m; k < g.n_rows; k++) o[k] = -1;
    }
    free(bins);
    return 0;
}

/* S6  Track selection: candidates in priority order (more hits first, then smaller chain start)
 * keep the hits no already-accepted candidate owns; a candidate keeping at least N_MIN hits is
 * accepted and owns them.  seg_hits/seg_n hold the kept hits (ascending rows). */
typedef struct { int32_t n, start, idx; } or_prio;
static int prio_cmp(const void *a, const void *b) {
    const or_prio *x = (const or_prio *)a, *y = (const or_prio *)b;
    if (x->n != y->n) return x->n > y->n ? -1 : 1;
    if (x->start != y->start) return x->start < y->start ? -1 : 1;
    return 0;
}
int or_select(int32_t n, int32_t n_rows, int32_t n_cand, const int32_t *cand_hits, const int32_t *cand_n,
              const int32_t *cand_start, int32_t *seg_hits, int32_t *seg_n, int32_t *accepted) {
    or_prio *pr = (or_prio *)malloc(sizeof(or_prio) * (n_cand > 0 ? n_cand : 1));
    for (int32_t t = 0; t < n_cand; t++) { pr[t].n = cand_n[t]; pr[t].start = cand_start[t]; pr[t].idx = t; }
    qsort(pr, n_cand, sizeof(or_prio), prio_cmp);
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (int32_t c = 0; c < n; c++) owner[c] = -1;
    for (int32_t t = 0; t < n_cand; t++) { accepted[t] = 0; seg_n[t] = 0; }
    for (int32_t i = 0; i < n_cand; i++) {
        int32_t t = pr[i].idx;
        const int32_t *h = cand_hits + (int64_t)t * n_rows;
        int32_t *o = seg_hits + (int64_t)t * n_rows;
        int kept = 0;
        for (int k = 0; k < cand_n[t]; k++) if (owner[h[k]] < 0) o[kept++] = h[k];
        if (kept >= OR_N_MIN) {
            accepted[t] = 1;
            seg_n[t] = kept;
            for (int k = 0; k < kept; k++) owner[o[k]] = t;
        }
        for (int k = (accepted[t] ? kept : 0); k < n_rows; k++) o[k] = -1;
    }
    free(owner);
    free(pr);
    return 0;
}

/* S7  Inter-sector merge (section 3: sectors are tracked independently, segments merged after).
 * The outer end of segment S (its last kept hit and the hit MERGE_BACK positions earlier, in the
 * sector frame on integer (Xtab[row], Y) coordinates) is rotated into the frame of an adjacent
 * sector of the same side with the integer constants (C30, S30), extrapolated linearly to the
 * row of the first hit of segment T, and compared there.  Mutual best pairs (smallest
 * (D, index)) are linked S -> T.  next[] receives the links. */
/* The merge decision on integer coordinates.  (X1, Y1, Z1) and (X2, Y2, Z2) are the hit MERGE_BACK
 * positions before the outer end of S and its last hit, in the frame of S's sector ks; (XT, YT, ZT)
 * is T's first hit in the frame of its sector kt.  Returns 1 and *D_out on a match. */
static int merge_decide(const or_geom *g, int ks, int64_t X1, int64_t Y1, int64_t Z1, int64_t X2, int64_t Y2,
                        int64_t Z2, int kt, int64_t XT, int64_t YT, int64_t ZT, int64_t *D_out) {
    int half = g->n_sectors / 2;
    int hs_ = ks % half, ht_ = kt % half;
    int sgn;
    if ((ks < half) != (kt < half)) return 0;
    if ((hs_ + 1) % half == ht_) sgn = +1;           /* T is the next sector in phi      */
    else if ((ht_ + 1) % half == hs_) sgn = -1;      /* T is the previous sector in phi  */
    else return 0;
    int64_t x2 = floor_shift(X2 * g->c30 + sgn * Y2 * g->s30, 30);
    int64_t y2 = floor_shift(-sgn * X2 * g->s30 + Y2 * g->c30, 30);
    int64_t x1 = floor_shift(X1 * g->c30 + sgn * Y1 * g->s30, 30);
    int64_t y1 = floor_shift(-sgn * X1 * g->s30 + Y1 * g->c30, 30);
    int64_t dxs = x2 - x1;
    if (dxs <= 0) return 0;
    if (iabs64(XT - x2) > OR_MERGE_XMAX) return 0;
    int64_t yp = y1 + floor_div((XT - x1) * (y2 - y1), dxs);
    int64_t zp = Z1 + floor_div((XT - x1) * (Z2 - Z1), dxs);
    int64_t dy = YT - yp, dz = ZT - zp;
    if (iabs64(dy) > OR_W_MERGE || iabs64(dz) > OR_W_MERGE) return 0;
    *D_out = dy * dy + dz * dz;
    return 1;
}

static int merge_match(const or_geom *g, const int16_t *pad, const uint16_t *tim, const int32_t *bins,
                       const int32_t *hs, int ns, const int32_t *ht, int64_t *D_out) {
    int ks = bins[hs[ns - 1]] / g->n_rows, kt = bins[ht[0]] / g->n_rows;
    int32_t hL = hs[ns - 1], hB = hs[ns - 1 - OR_MERGE_BACK];
    return merge_decide(g, ks, g->xtab[bins[hB] % g->n_rows], pad[hB], tim[hB], g->xtab[bins[hL] % g->n_rows],
                        pad[hL], tim[hL], kt, g->xtab[bins[ht[0]] % g->n_rows], pad[ht[0]], tim[ht[0]], D_out);
}

int or_merge(const or_geom_in *gin, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off,
             int32_t n, int32_t n_seg, const int32_t *seg_hits, const int32_t *seg_n, const int32_t *gap_next,
             int32_t *next) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    /* with gap links (OR_RULE_GAP_MERGE) a segment that continues in its own sector is not an outer
     * end, and one that is continued from its own sector is not a first segment */
    char *gap_src = (char *)calloc((size_t)n_seg + 1, 1), *gap_dst = (char *)calloc((size_t)n_seg + 1, 1);
    if (gap_next)
        for (int32_t i = 0; i < n_seg; i++)
            if (gap_next[i] >= 0) { gap_src[i] = 1; gap_dst[gap_next[i]] = 1; }
    int nbins = g.n_sectors * g.n_rows;
    int32_t *bins = cluster_bins(bin_off, nbins, n);
    int64_t *bestT_D = (int64_t *)malloc(sizeof(int64_t) * (n_seg + 1));
    int32_t *bestT = (int32_t *)malloc(sizeof(int32_t) * (n_seg + 1));
    int64_t *bestS_D = (int64_t *)malloc(sizeof(int64_t) * (n_seg + 1));
    int32_t *bestS = (int32_t *)malloc(sizeof(int32_t) * (n_seg + 1));
    for (int32_t i = 0; i < n_seg; i++) { bestT[i] = -1; bestS[i] = -1; next[i] = -1; }
    /* segments listed per sector of their first hit (a segment never leaves its sector) */
    int32_t *sec_cnt = (int32_t *)calloc((size_t)g.n_sectors + 1, sizeof(int32_t));
    int32_t *sec_list = (int32_t *)malloc(sizeof(int32_t) * (n_seg + 1));
    for (int32_t s = 0; s < n_seg; s++)
        if (seg_n[s] >= OR_N_MIN) sec_cnt[bins[seg_hits[(int64_t)s * g.n_rows]] / g.n_rows + 1]++;
    for (int k = 0; k < g.n_sectors; k++) sec_cnt[k + 1] += sec_cnt[k];
    int32_t *fill = (int32_t *)calloc((size_t)g.n_sectors + 1, sizeof(int32_t));
    for (int32_t s = 0; s < n_seg; s++) {
        if (seg_n[s] < OR_N_MIN) continue;
        int k = bins[seg_hits[(int64_t)s * g.n_rows]] / g.n_rows;
        sec_list[sec_cnt[k] + fill[k]++] = s;
    }
    for (int32_t s = 0; s < n_seg; s++) {
        if (seg_n[s] < OR_N_MIN || gap_src[s]) continue;
        const int32_t *hs = seg_hits + (int64_t)s * g.n_rows;
        int ks = bins[hs[0]] / g.n_rows, half = g.n_sectors / 2;
        int side0 = ks < half ? 0 : half;
        for (int nb = 0; nb < 2; nb++) {
            int kt = side0 + ((ks - side0) + (nb == 0 ? 1 : half - 1)) % half;
            for (int32_t i = sec_cnt[kt]; i < sec_cnt[kt + 1]; i++) {
                int32_t t = sec_list[i];
                int64_t D;
                if (t == s || gap_dst[t]) continue;
                if (!merge_match(&g, pad, tim, bins, hs, seg_n[s], seg_hits + (int64_t)t * g.n_rows, &D)) continue;
                if (bestT[s] < 0 || D < bestT_D[s] || (D == bestT_D[s] && t < bestT[s])) { bestT[s] = t; bestT_D[s] = D; }
                if (bestS[t] < 0 || D < bestS_D[t] || (D == bestS_D[t] && s < bestS[t])) { bestS[t] = s; bestS_D[t] = D; }
            }
        }
    }
    free(sec_cnt); free(sec_list); free(fill);
    for (int32_t s = 0; s < n_seg; s++)
        if (bestT[s] >= 0 && bestS[bestT[s]] == s) next[s] = bestT[s];
    free(bestT_D); free(bestT); free(bestS_D); free(bestS); free(bins); free(gap_src); free(gap_dst);
    return 0;
}

/* S7' Gap merge inside a sector (OR_RULE_GAP_MERGE; section 3, segment merging, applied to the
 * segments of one sector that a gap of pad rows without clusters splits, e.g. dead rows).  The
 * integer filter of the following runs over the kept hits of segment S in ascending rows (one
 * step per row, an update per hit) and predicts on, row by row, up to OR_GAP_MAX rows past S's
 * last hit.  A segment T of the same sector whose first kept hit lies on one of those rows, k rows
 * past S's last hit, is a candidate when that hit is within the following's search radius after
 * k-1 misses, W_F0 + W_F1 (k-1), of the prediction: D = dY^2 + dZ^2 <= radius^2.  Mutual best
 * pairs by (D, index) are linked S -> T. */
int or_gap_merge(const or_geom_in *gin, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off,
                 int32_t n, int32_t n_seg, const int32_t *seg_hits, const int32_t *seg_n, int32_t *gap_next) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    int nbins = g.n_sectors * g.n_rows;
    int32_t *bins = cluster_bins(bin_off, nbins, n);
    int64_t *bestT_D = (int64_t *)malloc(sizeof(int64_t) * (n_seg + 1));
    int32_t *bestT = (int32_t *)malloc(sizeof(int32_t) * (n_seg + 1));
    int64_t *bestS_D = (int64_t *)malloc(sizeof(int64_t) * (n_seg + 1));
    int32_t *bestS = (int32_t *)malloc(sizeof(int32_t) * (n_seg + 1));
    for (int32_t i = 0; i < n_seg; i++) { bestT[i] = -1; bestS[i] = -1; gap_next[i] = -1; }
    /* accepted segments listed per bin of their first hit (sector, first row) */
    int32_t *cnt = (int32_t *)calloc((size_t)nbins + 1, sizeof(int32_t));
    int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (n_seg + 1));
    int32_t *fill = (int32_t *)calloc((size_t)nbins + 1, sizeof(int32_t));
    for (int32_t t = 0; t < n_seg; t++)
        if (seg_n[t] >= OR_N_MIN) cnt[bins[seg_hits[(int64_t)t * g.n_rows]] + 1]++;
    for (int k = 0; k < nbins; k++) cnt[k + 1] += cnt[k];
    for (int32_t t = 0; t < n_seg; t++) {
        if (seg_n[t] < OR_N_MIN) continue;
        int b = bins[seg_hits[(int64_t)t * g.n_rows]];
        list[cnt[b] + fill[b]++] = t;
    }
    /* backward filter of every accepted segment: over its kept hits in descending rows, the state
     * at its first hit */
    abg *back_y = (abg *)malloc(sizeof(abg) * (n_seg + 1)), *back_z = (abg *)malloc(sizeof(abg) * (n_seg + 1));
    for (int32_t t = 0; t < n_seg; t++) {
        if (seg_n[t] < OR_N_MIN) continue;
        const int32_t *ht = seg_hits + (int64_t)t * g.n_rows;
        int nt_ = seg_n[t];
        int64_t d = bins[ht[nt_ - 1]] % g.n_rows - bins[ht[nt_ - 2]] % g.n_rows;
        abg_init(&back_y[t], pad[ht[nt_ - 1]], pad[ht[nt_ - 2]], d);
        abg_init(&back_z[t], tim[ht[nt_ - 1]], tim[ht[nt_ - 2]], d);
        for (int k = nt_ - 2; k >= 0; k--) {
            for (int64_t j = bins[ht[k + 1]] % g.n_rows - bins[ht[k]] % g.n_rows; j > 0; j--) {
                abg_predict(&back_y[t]); abg_predict(&back_z[t]);
            }
            abg_update(&back_y[t], pad[ht[k]]); abg_update(&back_z[t], tim[ht[k]]);
        }
    }
    for (int32_t s = 0; s < n_seg; s++) {
        if (seg_n[s] < OR_N_MIN) continue;
        const int32_t *hs = seg_hits + (int64_t)s * g.n_rows;
        int ns = seg_n[s];
        int ks = bins[hs[0]] / g.n_rows;
        abg fy, fz;
        int64_t d01 = bins[hs[1]] % g.n_rows - bins[hs[0]] % g.n_rows;
        abg_init(&fy, pad[hs[0]], pad[hs[1]], d01);
        abg_init(&fz, tim[hs[0]], tim[hs[1]], d01);
        for (int k = 1; k < ns; k++) {
            for (int64_t j = bins[hs[k]] % g.n_rows - bins[hs[k - 1]] % g.n_rows; j > 0; j--) {
                abg_predict(&fy); abg_predict(&fz);
            }
            abg_update(&fy, pad[hs[k]]); abg_update(&fz, tim[hs[k]]);
        }
        int rs = bins[hs[ns - 1]] % g.n_rows;
        for (int rt = rs + 1; rt < g.n_rows && rt <= rs + OR_GAP_MAX; rt++) {
            abg_predict(&fy); abg_predict(&fz);
            int64_t py = q16_round(fy.p), pz = q16_round(fz.p);
            /* the stop rules of the following: a prediction that leaves the sector, the drift range
             * or the slope limit ends the search (the segment ended there, not in a gap) */
            if (iabs64(py) > g.ymax[rt] || pz < 0 || pz > g.zmax || iabs64(fy.v) > (int64_t)OR_V_MAX * 65536) break;
            if (rt - rs - 1 < OR_M_MISS) continue;      /* a shorter gap the following bridges */
            int64_t w = OR_W_F0 + (int64_t)OR_W_F1 * (rt - rs - 1);
            int b = ks * g.n_rows + rt;
            for (int32_t i = cnt[b]; i < cnt[b + 1]; i++) {
                int32_t t = list[i];
                if (t == s) continue;
                int32_t h = seg_hits[(int64_t)t * g.n_rows];
                int64_t dy = pad[h] - py, dz = tim[h] - pz;
                if (iabs64(dy) > w || iabs64(dz) > w || dy * dy + dz * dz > w * w) continue;
                /* and T's backward prediction at S's last row, rt - rs rows back */
                abg by = back_y[t], bz = back_z[t];
                int inside = 1;
                for (int j = 1; j <= rt - rs && inside; j++) {
                    abg_predict(&by); abg_predict(&bz);
                    int64_t qy = q16_round(by.p), qz = q16_round(bz.p);
                    inside = iabs64(qy) <= g.ymax[rt - j] && qz >= 0 && qz <= g.zmax &&
                             iabs64(by.v) <= (int64_t)OR_V_MAX * 65536;
                }
                if (!inside) continue;
                int64_t ey = pad[hs[ns - 1]] - q16_round(by.p), ez = tim[hs[ns - 1]] - q16_round(bz.p);
                if (iabs64(ey) > w || iabs64(ez) > w || ey * ey + ez * ez > w * w) continue;
                int64_t D = dy * dy + dz * dz + ey * ey + ez * ez;
                if (bestT[s] < 0 || D < bestT_D[s] || (D == bestT_D[s] && t < bestT[s])) { bestT[s] = t; bestT_D[s] = D; }
                if (bestS[t] < 0 || D < bestS_D[t] || (D == bestS_D[t] && s < bestS[t])) { bestS[t] = s; bestS_D[t] = D; }
            }
        }
    }
    for (int32_t s = 0; s < n_seg; s++)
        if (bestT[s] >= 0 && bestS[bestT[s]] == s) gap_next[s] = bestT[s];
    free(cnt); free(list); free(fill); free(back_y); free(back_z);
    free(bestT_D); free(bestT); free(bestS_D); free(bestS); free(bins);
    return 0;
}

/* Assemble merged tracks: one track per chain of linked segments, ordered by the index of its
 * first segment; a cycle of links is cut in front of its smallest segment.  Writes trk_off
 * (n_trk+1), trk_hits and label (track id or -1).  Returns the number of tracks or -2. */
int32_t or_assemble(int32_t n, int32_t n_rows, int32_t n_seg, const int32_t *seg_hits, const int32_t *seg_n,
                    const int32_t *next_in, int32_t *trk_off, int32_t *trk_hits, int32_t *label,
                    int32_t cap_trk, int32_t cap_hits) {
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (n_seg + 1));
    int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * (n_seg + 1));
    char *seen = (char *)calloc(n_seg + 1, 1);
    for (int32_t i = 0; i < n_seg; i++) { next[i] = next_in[i]; prev[i] = -1; }
    for (int32_t i = 0; i < n_seg; i++) if (next[i] >= 0) prev[next[i]] = i;
    for (int32_t i = 0; i < n_seg; i++) {
        if (seg_n[i] < OR_N_MIN || prev[i] >= 0) continue;
        for (int32_t x = i; x >= 0; x = next[x]) seen[x] = 1;
    }
    for (int32_t i = 0; i < n_seg; i++) {
        if (seg_n[i] < OR_N_MIN || seen[i]) continue;
        int32_t m = i;
        for (int32_t x = next[i]; x != i; x = next[x]) if (x < m) m = x;
        next[prev[m]] = -1;
        prev[m] = -1;
        for (int32_t x = m; x >= 0; x = next[x]) seen[x] = 1;
    }
    for (int32_t c = 0; c < n; c++) label[c] = -1;
    int32_t nt = 0, nh = 0;
    trk_off[0] = 0;
    for (int32_t i = 0; i < n_seg; i++) {
        if (seg_n[i] < OR_N_MIN || prev[i] >= 0) continue;
        if (nt >= cap_trk) { nt = -2; break; }
        for (int32_t x = i; x >= 0; x = next[x]) {
            for (int k = 0; k < seg_n[x]; k++) {
                if (nh >= cap_hits) { nt = -2; goto done; }
                int32_t c = seg_hits[(int64_t)x * n_rows + k];
                trk_hits[nh++] = c;
                label[c] = nt;
            }
        }
        nt++;
        trk_off[nt] = nh;
    }
done:
    free(next); free(prev); free(seen);
    return nt;
}

/* S11  Time-frame slice merge (section 3, its outlook for continuous readout: a time frame is cut
 * along the drift-time axis, the slices are tracked one by one, and the track segments are merged
 * afterwards).  The clusters are those of n_slices consecutive slices of slice_len LSB of readout
 * time, with slice-local times, in the layout of a batch of events (bin = (slice, sector, row));
 * the tracks are the per-slice tracking output in slice order (ev_trk_off[j] = first track of
 * slice j), hits in track order.
 *
 * A track keeps a readout time that falls outwards (drift length shrinks as |z| grows), so the
 * piece of a track in slice j+1 (S) ends, at its outer end, where the piece in slice j (T)
 * begins.  The outer end of S (its last hit and the hit MERGE_BACK positions earlier, on integer
 * (Xtab[row], Y, Z)), with the times moved into slice j by + slice_len, is extrapolated linearly
 * (floor division) to the row of T's first hit and compared there with the merge windows.  T's
 * first hit lies in the sector of S's last hit, or in an adjacent sector of the same side; then
 * the end of S is first rotated into T's frame exactly as in the inter-sector merge.  Mutual best
 * pairs (smallest (D, index) on both sides) are linked S -> T. */
static int frame_match(const or_geom *g, const int16_t *pad, const uint16_t *tim, const int32_t *bins,
                       int32_t slice_len, const int32_t *hs, int ns, int32_t hT, int64_t *D_out) {
    const int nbe = g->n_sectors * g->n_rows, half = g->n_sectors / 2;
    int32_t hL = hs[ns - 1], hB = hs[ns - 1 - OR_MERGE_BACK];
    int ks = (bins[hL] % nbe) / g->n_rows, kt = (bins[hT] % nbe) / g->n_rows;
    int sgn;
    if ((ks < half) != (kt < half)) return 0;
    if (ks == kt) sgn = 0;                                        /* same sector            */
    else if ((ks % half + 1) % half == kt % half) sgn = +1;       /* T in the next sector   */
    else if ((kt % half + 1) % half == ks % half) sgn = -1;       /* T in the previous one  */
    else return 0;
    int64_t X2 = g->xtab[bins[hL] % g->n_rows], Y2 = pad[hL], Z2 = (int64_t)tim[hL] + slice_len;
    int64_t X1 = g->xtab[bins[hB] % g->n_rows], Y1 = pad[hB], Z1 = (int64_t)tim[hB] + slice_len;
    int64_t x1 = X1, y1 = Y1, x2 = X2, y2 = Y2;
    if (sgn != 0) {
        x2 = floor_shift(X2 * g->c30 + sgn * Y2 * g->s30, 30);
        y2 = floor_shift(-sgn * X2 * g->s30 + Y2 * g->c30, 30);
        x1 = floor_shift(X1 * g->c30 + sgn * Y1 * g->s30, 30);
        y1 = floor_shift(-sgn * X1 * g->s30 + Y1 * g->c30, 30);
    }
    int64_t XT = g->xtab[bins[hT] % g->n_rows], YT = pad[hT], ZT = tim[hT];
    int64_t dxs = x2 - x1;
    if (dxs <= 0) return 0;
    if (iabs64(XT - x2) > OR_MERGE_XMAX) return 0;
    int64_t yp = y1 + floor_div((XT - x1) * (y2 - y1), dxs);
    int64_t zp = Z1 + floor_div((XT - x1) * (Z2 - Z1), dxs);
    int64_t dy = YT - yp, dz = ZT - zp;
    if (iabs64(dy) > OR_W_MERGE || iabs64(dz) > OR_W_MERGE) return 0;
    *D_out = dy * dy + dz * dz;
    return 1;
}

int or_frame_merge(const or_geom_in *gin, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off,
                   int32_t n, int32_t n_slices, int32_t slice_len, int32_t n_trk, const int32_t *trk_off,
                   const int32_t *trk_hits, const int32_t *ev_trk_off, int32_t *next) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    if (n_slices < 1 || slice_len < 1) return -1;
    int32_t *bins = cluster_bins(bin_off, n_slices * g.n_sectors * g.n_rows, n);
    int64_t *bestT_D = (int64_t *)malloc(sizeof(int64_t) * (n_trk + 1));
    int32_t *bestT = (int32_t *)malloc(sizeof(int32_t) * (n_trk + 1));
    int64_t *bestS_D = (int64_t *)malloc(sizeof(int64_t) * (n_trk + 1));
    int32_t *bestS = (int32_t *)malloc(sizeof(int32_t) * (n_trk + 1));
    for (int32_t i = 0; i < n_trk; i++) { bestT[i] = -1; bestS[i] = -1; next[i] = -1; }
    for (int j = 0; j + 1 < n_slices; j++) {
        for (int32_t s = ev_trk_off[j + 1]; s < ev_trk_off[j + 2]; s++) {
            int ns = trk_off[s + 1] - trk_off[s];
            if (ns <= OR_MERGE_BACK) continue;
            const int32_t *hs = trk_hits + trk_off[s];
            for (int32_t t = ev_trk_off[j]; t < ev_trk_off[j + 1]; t++) {
                int64_t D;
                if (trk_off[t + 1] <= trk_off[t]) continue;
                if (!frame_match(&g, pad, tim, bins, slice_len, hs, ns, trk_hits[trk_off[t]], &D)) continue;
                if (bestT[s] < 0 || D < bestT_D[s] || (D == bestT_D[s] && t < bestT[s])) { bestT[s] = t; bestT_D[s] = D; }
                if (bestS[t] < 0 || D < bestS_D[t] || (D == bestS_D[t] && s < bestS[t])) { bestS[t] = s; bestS_D[t] = D; }
            }
        }
    }
    for (int32_t s = 0; s < n_trk; s++)
        if (bestT[s] >= 0 && bestS[bestT[s]] == s) next[s] = bestT[s];
    free(bestT_D); free(bestT); free(bestS_D); free(bestS); free(bins);
    return 0;
}

/* Frame tracks: one per chain of linked slice tracks, ordered by the index of the chain's first
 * track; hits in chain order (links only go from slice j+1 to slice j, so there is no cycle).
 * Writes ftrk_off (n_ftrk+1), ftrk_hits and flabel (frame track id or -1).  Returns n_ftrk, or -2
 * when a capacity is exceeded. */
int32_t or_frame_assemble(int32_t n, int32_t n_trk, const int32_t *trk_off, const int32_t *trk_hits,
                          const int32_t *next, int32_t *ftrk_off, int32_t *ftrk_hits, int32_t *flabel,
                          int32_t cap_trk, int32_t cap_hits) {
    char *has_prev = (char *)calloc(n_trk + 1, 1);
    for (int32_t i = 0; i < n_trk; i++) if (next[i] >= 0) has_prev[next[i]] = 1;
    for (int32_t c = 0; c < n; c++) flabel[c] = -1;
    int32_t nt = 0, nh = 0;
    ftrk_off[0] = 0;
    for (int32_t i = 0; i < n_trk; i++) {
        if (has_prev[i]) continue;
        if (nt >= cap_trk) { nt = -2; break; }
        for (int32_t x = i; x >= 0; x = next[x]) {
            for (int32_t k = trk_off[x]; k < trk_off[x + 1]; k++) {
                if (nh >= cap_hits) { nt = -2; goto done; }
                ftrk_hits[nh++] = trk_hits[k];
                flabel[trk_hits[k]] = nt;
            }
        }
        nt++;
        ftrk_off[nt] = nh;
    }
done:
    free(has_prev);
    return nt;
}

/* ============================================================================================
 * S0 / S8  Cluster transformation and Kalman-filter track refit in double precision.
 * Transform (calibration theta = [s_vd, d_0..d_{ns-1}, a_0..a_{ns-1}]), for a cluster of sector k
 * and row r with raw y = Y*lsb and drift length D = Z*lsb:
 *   z = side*(z_max - s_vd*D) + d_k,  (x, y) = (x_r, y)*(1 + a_k*(rho - x_first)/(span*rho)),
 * rho = |(x_r, y)|.  The fit runs from the last hit of the track to the first, with the local
 * helix state (y, z, sin phi, tan lambda, q/pT) at x in the frame of the current hit's sector.
 * ========================================================================================== */
/* A point under calibration theta; jy, jz = factors by which the transformation scales a raw
 * y and z error (1 + a_k g(rho) and s_vd; the change of g across a pad row is neglected). */
typedef struct { double x, y, z, jy, jz; } or_pt;

static double sector_alpha(const or_geom *g, int k) { return ((k % (g->n_sectors / 2)) + 0.5) * 2.0 * g->half_angle; }

static or_pt transform(const or_geom *g, double x_first, double span, int k, int r, int64_t Y, int64_t Z,
                       const double *th) {
    int ns = g->n_sectors;
    double side = k < ns / 2 ? 1.0 : -1.0;
    double xr = g->xr[r], y = (double)Y * g->lsb, D = (double)Z * g->lsb;
    or_pt p;
    p.z = side * (g->z_max - th[0] * D) + th[1 + k];
    double rho = sqrt(xr * xr + y * y);
    double sc = 1.0 + th[1 + ns + k] * (rho - x_first) / (span * rho);
    p.x = xr * sc;
    p.y = y * sc;
    p.jy = sc;
    p.jz = th[0];
    return p;
}

/* asin(u)/u, with its limit 1 at u = 0 */
static double asinc(double u) { return fabs(u) < 1e-8 ? 1.0 + u * u / 6.0 : asin(u) / u; }

/* 5x5 helpers on full matrices */
static void mat_FPFt(double P[5][5], double F[5][5]) {
    double T[5][5], R[5][5];
    for (int i = 0; i < 5; i++) for (int j = 0; j < 5; j++) {
        double s = 0; for (int k = 0; k < 5; k++) s += F[i][k] * P[k][j]; T[i][j] = s;
    }
    for (int i = 0; i < 5; i++) for (int j = 0; j < 5; j++) {
        double s = 0; for (int k = 0; k < 5; k++) s += T[i][k] * F[j][k]; R[i][j] = s;
    }
    memcpy(P, R, sizeof(R));
}

typedef struct {
    double x, p[5], P[5][5];
    int frame;
    double chi2;
    int ok;
} or_kf;

/* Rotate the state into the frame of sector k_new (reference surface moved with the point). */
static void kf_rotate(const or_geom *g, or_kf *s, int k_new) {
    double da = sector_alpha(g, k_new) - sector_alpha(g, s->frame);
    while (da > OR_PI) da -= 2 * OR_PI;
    while (da <= -OR_PI) da += 2 * OR_PI;
    double ca = cos(da), sa = sin(da);
    double sn = s->p[2], cs = sqrt(1.0 - sn * sn);
    double x1 = s->x * ca + s->p[0] * sa;
    double y1 = -s->x * sa + s->p[0] * ca;
    double sn1 = sn * ca - cs * sa;
    double cs1 = cs * ca + sn * sa;
    if (cs1 <= OR_CPHI_MIN) { s->ok = 0; return; }
    double C = g->kB * s->p[4];
    double J[5][5] = {{0}};
    for (int i = 0; i < 5; i++) J[i][i] = 1.0;
    J[0][0] = cs / cs1;
    J[1][0] = -s->p[3] * sa / cs1;
    J[2][0] = -C * sa;
    J[2][2] = cs1 / cs;
    mat_FPFt(s->P, J);
    s->x = x1;
    s->p[0] = y1;
    s->p[2] = sn1;
    s->frame = k_new;
}

/* Helix step from local x to xh (section 3, the track following; exact in the state): with C = kB q/pT,
 * sin phi2 = sin phi + C dx, dy = dx (sin phi + sin phi2)/(cos phi + cos phi2), chord
 * L = dx sqrt(1 + T^2), arc = L asin(C L/2)/(C L/2), dz = tan lambda * arc.  F is the step Jacobian
 * d(state')/d(state), written in terms of T = tan of the mean direction (the derivatives of dz keep
 * the leading chord term).  Returns 0 when |sin phi| reaches the parametrisation limit. */
static int prop_step(const or_geom *g, double x, const double *p, double xh, double *po, double F[5][5]) {
    double dx = xh - x;
    double sn = p[2], tl = p[3], q = p[4];
    double C = g->kB * q;
    double sn2 = sn + C * dx;
    if (fabs(sn2) >= OR_SNP_MAX || fabs(sn) >= OR_SNP_MAX) return 0;
    double c1 = sqrt(1.0 - sn * sn), c2 = sqrt(1.0 - sn2 * sn2);
    double T = (sn + sn2) / (c1 + c2);
    double W = 1.0 + T * T, sW = sqrt(W);
    double L = dx * sW;
    double arc = L * asinc(0.5 * C * L);
    double h = 0.5 * (1.0 / c1 + 1.0 / c2);
    double g2 = 0.5 / c2 * g->kB * dx * dx;
    for (int i = 0; i < 5; i++) for (int j = 0; j < 5; j++) F[i][j] = i == j ? 1.0 : 0.0;
    F[0][2] = dx * W * h;
    F[0][4] = W * g2;
    F[1][2] = tl * dx * T * sW * h;
    F[1][3] = arc;
    F[1][4] = tl * T * sW * g2;
    F[2][4] = g->kB * dx;
    po[0] = p[0] + dx * T;
    po[1] = p[1] + tl * arc;
    po[2] = sn2;
    po[3] = tl;
    po[4] = q;
    return 1;
}

static void kf_propagate(const or_geom *g, or_kf *s, double xh) {
    double F[5][5], po[5];
    if (!prop_step(g, s->x, s->p, xh, po, F)) { s->ok = 0; return; }
    mat_FPFt(s->P, F);
    for (int i = 0; i < 5; i++) s->p[i] = po[i];
    s->x = xh;
}

/* Measurement update with (y, z) of variances (vy, vz): gain K = P H^T S^-1, P <- (I - K H) P
 * then symmetrised. */
static void kf_update(or_kf *s, double ym, double zm, double vy, double vz) {
    double r0 = ym - s->p[0], r1 = zm - s->p[1];
    double S00 = s->P[0][0] + vy, S01 = s->P[0][1], S11 = s->P[1][1] + vz;
    double det = S00 * S11 - S01 * S01;
    double i00 = S11 / det, i01 = -S01 / det, i11 = S00 / det;
    s->chi2 += r0 * r0 * i00 + 2.0 * r0 * r1 * i01 + r1 * r1 * i11;
    double K[5][2];
    for (int i = 0; i < 5; i++) {
        K[i][0] = s->P[i][0] * i00 + s->P[i][1] * i01;
        K[i][1] = s->P[i][0] * i01 + s->P[i][1] * i11;
    }
    for (int i = 0; i < 5; i++) s->p[i] += K[i][0] * r0 + K[i][1] * r1;
    double A[5][5];
    for (int i = 0; i < 5; i++) for (int j = 0; j < 5; j++)
        A[i][j] = s->P[i][j] - (K[i][0] * s->P[0][j] + K[i][1] * s->P[1][j]);
    for (int i = 0; i < 5; i++) for (int j = 0; j < 5; j++) s->P[i][j] = 0.5 * (A[i][j] + A[j][i]);
}

/* Seed at the last hit from the circle through the first, middle and last hit (nominal
 * coordinates, frame of the last hit's sector): signed curvature from the three points, the
 * tangent at the last hit from the chord direction plus half the turning angle, tan lambda from
 * dz over the arc length. */
static int kf_seed(const or_geom *g, const or_pt *pa, int ka, const or_pt *pb, int kb, const or_pt *pe, int ke,
                   double out[5]) {
    double ae = sector_alpha(g, ke);
    or_pt q[3];
    const or_pt *src[3] = {pa, pb, pe};
    int ks[3] = {ka, kb, ke};
    for (int i = 0; i < 3; i++) {
        double d = sector_alpha(g, ks[i]) - ae;
        q[i].x = src[i]->x * cos(d) - src[i]->y * sin(d);
        q[i].y = src[i]->x * sin(d) + src[i]->y * cos(d);
        q[i].z = src[i]->z;
    }
    double abx = q[1].x - q[0].x, aby = q[1].y - q[0].y;
    double bex = q[2].x - q[1].x, bey = q[2].y - q[1].y;
    double aex = q[2].x - q[0].x, aey = q[2].y - q[0].y;
    double lab = hypot(abx, aby), lbe = hypot(bex, bey), lae = hypot(aex, aey);
    if (lab <= 0 || lbe <= 0 || lae <= 0) return 0;
    double kappa = 2.0 * (abx * bey - aby * bex) / (lab * lbe * lae);
    double u = 0.5 * kappa * lae;
    if (fabs(u) >= 1.0) return 0;
    double phi = atan2(aey, aex) + asin(u);
    double arc = lae * asinc(u);
    out[0] = q[2].y;
    out[1] = q[2].z;
    out[2] = sin(phi);
    out[3] = (q[2].z - q[0].z) / arc;
    out[4] = kappa / g->kB;
    if (fabs(out[2]) >= OR_SNP_MAX) return 0;
    return 1;
}

/* Prior covariance of the seed state: sigma = 1 cm (y, z), 0.1 (sin phi, tan lambda), 1 c/GeV (q/pT).
 * Weak against the data of a track (posterior sigmas ~0.05 cm, ~1e-3, ~1e-2 c/GeV), and a
 * dynamic range an FP32 filter can carry (the refit on the GPU is FP32). */
static const double OR_C0[5] = {1.0, 1.0, 0.01, 0.01, 1.0};

/* Fit given points: measurements m[i] in the frame of sector ks[i] (hit order of the track).  The
 * seed takes sin phi, tan lambda and q/pT from the circle through the nominal points a, b, e
 * (first, middle, last hit) and its position from the last measurement.  Returns 1 on success.
 * mode 0: measurement errors sigma in y and z (the fit of section 3).  mode 1: errors sigma in
 * the raw coordinates, carried into the calibrated ones by the transformation (sigma jy,
 * sigma jz); chi2 is then -2 log L up to a theta-independent constant for raw errors that are
 * Gaussian with fixed sigma, and a change of theta that only rescales the data leaves it
 * unchanged (with fixed calibrated errors, shrinking the data would lower chi2). */
static int fit_points(const or_geom *g, int nh, const int *ks, const or_pt *m, const or_pt *a, const or_pt *b,
                      const or_pt *e, int mode, or_kf *s) {
    memset(s, 0, sizeof(*s));
    if (!kf_seed(g, a, ks[0], b, ks[(nh - 1) / 2], e, ks[nh - 1], s->p)) return 0;
    /* direction and curvature from the nominal circle; position at the last measurement itself */
    s->x = m[nh - 1].x;
    s->p[0] = m[nh - 1].y;
    s->p[1] = m[nh - 1].z;
    s->frame = ks[nh - 1];
    s->ok = 1;
    for (int i = 0; i < 5; i++) s->P[i][i] = OR_C0[i];
    for (int i = nh - 1; i >= 0; i--) {
        if (ks[i] != s->frame) kf_rotate(g, s, ks[i]);
        if (!s->ok) return 0;
        kf_propagate(g, s, m[i].x);
        if (!s->ok) return 0;
        if (mode == 1) {
            double vy = OR_SIGMA2 * m[i].jy * m[i].jy, vz = OR_SIGMA2 * m[i].jz * m[i].jz;
            kf_update(s, m[i].y, m[i].z, vy, vz);
        } else {
            kf_update(s, m[i].y, m[i].z, OR_SIGMA2, OR_SIGMA2);
        }
    }
    return 1;
}

/* General measurement update with d <= 3 components idx[] of the state, measured values m[] and
 * independent errors sig[]: S = H P H^T + R, K = P H^T S^-1, chi2 += r^T S^-1 r, p += K r,
 * P <- (I - K H) P, symmetrised.  S^-1 by Gauss-Jordan elimination with partial pivoting. */
static int kf_update_h(or_kf *s, int d, const int *idx, const double *m, const double *sig) {
    double S[3][6], r[3];
    for (int a = 0; a < d; a++) {
        r[a] = m[a] - s->p[idx[a]];
        for (int b = 0; b < d; b++) {
            S[a][b] = s->P[idx[a]][idx[b]] + (a == b ? sig[a] * sig[a] : 0.0);
            S[a][d + b] = a == b ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < d; c++) {
        int piv = c;
        for (int a = c + 1; a < d; a++) if (fabs(S[a][c]) > fabs(S[piv][c])) piv = a;
        if (S[piv][c] == 0.0) return 0;
        if (piv != c) for (int b = 0; b < 2 * d; b++) { double t = S[c][b]; S[c][b] = S[piv][b]; S[piv][b] = t; }
        double iv = 1.0 / S[c][c];
        for (int b = 0; b < 2 * d; b++) S[c][b] *= iv;
        for (int a = 0; a < d; a++) {
            if (a == c) continue;
            double f = S[a][c];
            for (int b = 0; b < 2 * d; b++) S[a][b] -= f * S[c][b];
        }
    }
    double Si[3][3];
    for (int a = 0; a < d; a++) for (int b = 0; b < d; b++) Si[a][b] = S[a][d + b];
    for (int a = 0; a < d; a++) for (int b = 0; b < d; b++) s->chi2 += r[a] * Si[a][b] * r[b];
    double K[5][3];
    for (int i = 0; i < 5; i++) for (int b = 0; b < d; b++) {
        double v = 0.0;
        for (int a = 0; a < d; a++) v += s->P[i][idx[a]] * Si[a][b];
        K[i][b] = v;
    }
    for (int i = 0; i < 5; i++) for (int b = 0; b < d; b++) s->p[i] += K[i][b] * r[b];
    double A[5][5];
    for (int i = 0; i < 5; i++) for (int j = 0; j < 5; j++) {
        double v = s->P[i][j];
        for (int b = 0; b < d; b++) v -= K[i][b] * s->P[idx[b]][j];
        A[i][j] = v;
    }
    for (int i = 0; i < 5; i++) for (int j = 0; j < 5; j++) s->P[i][j] = 0.5 * (A[i][j] + A[j][i]);
    return 1;
}

/* Reference measurements at the production vertex (reading of the drift calibration by matching
 * TPC tracks to inner-tracker tracks, section 6).  ref[8] of one track: ref[0] = sigma_v of the
 * vertex point (y, z) = (0, 0) at x = 0 in the frame of the first hit's sector; (ref[1], ref[2]) =
 * (z0, sigma), (ref[3], ref[4]) = (tan lambda, sigma), (ref[5], ref[6]) = (q/pT, sigma) of the
 * reference track at the vertex; a sigma <= 0 leaves its term out, ref[7] is unused.  The state
 * at the first hit is propagated to x = 0 (exact helix step), updated with the vertex point, then
 * with the reference track's (z0, tan lambda, q/pT).  Returns 0 if the propagation fails. */
static int kf_anchor(const or_geom *g, or_kf *s, const double *ref) {
    int any = ref[0] > 0.0 || ref[2] > 0.0 || ref[4] > 0.0 || ref[6] > 0.0;
    if (!any) return 1;
    kf_propagate(g, s, 0.0);
    if (!s->ok) return 0;
    if (ref[0] > 0.0) {
        int idx[2] = {0, 1};
        double m[2] = {0.0, 0.0}, sg[2] = {ref[0], ref[0]};
        if (!kf_update_h(s, 2, idx, m, sg)) return 0;
    }
    int idx[3], d = 0;
    double m[3], sg[3];
    const int comp[3] = {1, 3, 4};
    for (int c = 0; c < 3; c++)
        if (ref[2 + 2 * c] > 0.0) { idx[d] = comp[c]; m[d] = ref[1 + 2 * c]; sg[d] = ref[2 + 2 * c]; d++; }
    if (d > 0 && !kf_update_h(s, d, idx, m, sg)) return 0;
    return 1;
}

/* Fit one track from its raw clusters: measurements transformed with theta, seed points with the
 * nominal calibration (the seed does not depend on theta). */
static int fit_track(const or_geom *g, double x_first, double span, const int16_t *pad, const uint16_t *tim,
                     const int32_t *bins, const int32_t *hits, int nh, const double *theta, int mode, or_kf *s) {
    double th0[1 + 2 * 64] = {0.0};
    th0[0] = 1.0;
    int nr = g->n_rows;
    int ks[OR_MAX_ROWS * 4];
    or_pt m[OR_MAX_ROWS * 4];
    if (nh > OR_MAX_ROWS * 4) return 0;
    for (int i = 0; i < nh; i++) {
        int k = bins[hits[i]] / nr, r = bins[hits[i]] % nr;
        ks[i] = k;
        m[i] = transform(g, x_first, span, k, r, pad[hits[i]], tim[hits[i]], theta);
    }
    int ib = (nh - 1) / 2;
    or_pt a = transform(g, x_first, span, ks[0], bins[hits[0]] % nr, pad[hits[0]], tim[hits[0]], th0);
    or_pt b = transform(g, x_first, span, ks[ib], bins[hits[ib]] % nr, pad[hits[ib]], tim[hits[ib]], th0);
    or_pt e = transform(g, x_first, span, ks[nh - 1], bins[hits[nh - 1]] % nr, pad[hits[nh - 1]], tim[hits[nh - 1]], th0);
    return fit_points(g, nh, ks, m, &a, &b, &e, mode, s);
}

/* S8: fit all tracks.  par[t*5] = (y, z, sin phi, tan lambda, q/pT) at xref[t] in the frame of the
 * first hit's sector; cov[t*15] lower triangle row-major; chi2, ndf = 2n-5 (0 and zeros if the
 * fit failed). */
int or_fit(const or_geom_in *gin, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off, int32_t n,
           int32_t n_trk, const int32_t *trk_off, const int32_t *trk_hits, const double *theta,
           double *par, double *xref, double *cov, double *chi2, int32_t *ndf) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    if (g.n_sectors > 64) return -1;
    int32_t *bins = cluster_bins(bin_off, g.n_sectors * g.n_rows, n);
    double span = gin->x_last - gin->x_first;
    for (int32_t t = 0; t < n_trk; t++) {
        or_kf s;
        int nh = trk_off[t + 1] - trk_off[t];
        int ok = nh >= 3 && fit_track(&g, gin->x_first, span, pad, tim, bins, trk_hits + trk_off[t], nh, theta, 0, &s);
        for (int i = 0; i < 5; i++) par[t * 5 + i] = ok ? s.p[i] : 0.0;
        int m = 0;
        for (int i = 0; i < 5; i++) for (int j = 0; j <= i; j++) cov[t * 15 + m++] = ok ? s.P[i][j] : 0.0;
        xref[t] = ok ? s.x : 0.0;
        chi2[t] = ok ? s.chi2 : 0.0;
        ndf[t] = ok ? 2 * nh - 5 : 0;
    }
    free(bins);
    return 0;
}

/* S9 reference: weighted sum of chi2 over the tracks that fit, at calibration theta.  weight may be
 * NULL (all 1); ref (may be NULL) adds each track's reference measurements at the vertex (see
 * kf_anchor; a track whose propagation to the vertex fails contributes nothing); mode selects the
 * measurement model (see fit_points: 0 fixed errors, 1 raw errors carried through the
 * transformation); `use` (may be NULL) restricts the sum to flagged tracks (used by the differences below,
 * which only refit the tracks a parameter can change). */
static double chi2_sum(const or_geom *g, double x_first, double span, const int16_t *pad, const uint16_t *tim,
                       const int32_t *bins, int32_t n_trk, const int32_t *trk_off, const int32_t *trk_hits,
                       const double *weight, const double *ref, int mode, const char *use, const double *theta) {
    double sum = 0.0;
    for (int32_t t = 0; t < n_trk; t++) {
        if (use && !use[t]) continue;
        const double w = weight ? weight[t] : 1.0;
        if (w == 0.0) continue;
        or_kf s;
        int nh = trk_off[t + 1] - trk_off[t];
        if (nh >= 3 && fit_track(g, x_first, span, pad, tim, bins, trk_hits + trk_off[t], nh, theta, mode, &s) &&
            (!ref || kf_anchor(g, &s, ref + 8 * (size_t)t)))
            sum += w * s.chi2;
    }
    return sum;
}

double or_chi2_total(const or_geom_in *gin, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off,
                     int32_t n, int32_t n_trk, const int32_t *trk_off, const int32_t *trk_hits, const double *weight,
                     const double *ref, int32_t mode, const double *theta) {
    or_geom g;
    if (make_geom(gin, &g)) return -1.0;
    int32_t *bins = cluster_bins(bin_off, g.n_sectors * g.n_rows, n);
    double v = chi2_sum(&g, gin->x_first, gin->x_last - gin->x_first, pad, tim, bins, n_trk, trk_off, trk_hits,
                        weight, ref, mode, NULL, theta);
    free(bins);
    return v;
}

/* Gradient of the weighted chi2 sum by central differences in double precision: the plain
 * definition of the derivative.  Steps h[0] (s_vd), h[1] (d_k), h[2] (a_k).  Only tracks touching
 * the perturbed sector are refitted for d_k and a_k (the others do not depend on them). */
int or_grad_fd(const or_geom_in *gin, const int16_t *pad, const uint16_t *tim, const int32_t *bin_off, int32_t n,
               int32_t n_trk, const int32_t *trk_off, const int32_t *trk_hits, const double *weight,
               const double *ref, int32_t mode, const double *theta, const double *h, double *grad) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    int ns = g.n_sectors, np = 1 + 2 * ns;
    int32_t *bins = cluster_bins(bin_off, ns * g.n_rows, n);
    double span = gin->x_last - gin->x_first;
    double *th = (double *)malloc(sizeof(double) * np);
    char *use = (char *)malloc(n_trk + 1);
    for (int j = 0; j < np; j++) {
        int sec = j == 0 ? -1 : (j - 1) % ns;
        double hj = j == 0 ? h[0] : (j <= ns ? h[1] : h[2]);
        for (int32_t t = 0; t < n_trk; t++) {
            use[t] = sec < 0;
            if (sec >= 0)
                for (int32_t i = trk_off[t]; i < trk_off[t + 1]; i++)
                    if (bins[trk_hits[i]] / g.n_rows == sec) { use[t] = 1; break; }
        }
        memcpy(th, theta, sizeof(double) * np);
        th[j] = theta[j] + hj;
        double fp = chi2_sum(&g, gin->x_first, span, pad, tim, bins, n_trk, trk_off, trk_hits, weight, ref, mode, use, th);
        th[j] = theta[j] - hj;
        double fm = chi2_sum(&g, gin->x_first, span, pad, tim, bins, n_trk, trk_off, trk_hits, weight, ref, mode, use, th);
        grad[j] = (fp - fm) / (2.0 * hj);
    }
    free(th); free(use); free(bins);
    return 0;
}

/* Reading constants, exported so that a test can compare them with the CUDA library's. */
int or_rule_constants(int64_t *out, int cap) {
    const int64_t v[] = {OR_RULE_SKIP_ROW, OR_RULE_GAP_MERGE, OR_GAP_MAX};
    int n = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < n && i < cap; i++) out[i] = v[i];
    return n;
}

int or_constants(int64_t *out, int cap) {
    int64_t v[] = {OR_W_LINK, OR_D_MAX, OR_N_SEED, OR_M_MISS, OR_W_F0, OR_W_F1, OR_V_MAX, OR_N_MIN,
                   OR_W_MERGE, OR_MERGE_XMAX, OR_MERGE_BACK};
    int nv = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < nv && i < cap; i++) out[i] = v[i];
    return nv;
}

/* ---- entry points used only by the pins (direct access to single steps) ------------------- */

/* S0 alone: transformed (x, y, z) of n clusters given their sector, row and raw coordinates. */
int or_transform(const or_geom_in *gin, int32_t n, const int32_t *sector, const int32_t *row, const int16_t *pad,
                 const uint16_t *tim, const double *theta, double *xyz) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    for (int32_t i = 0; i < n; i++) {
        or_pt p = transform(&g, gin->x_first, gin->x_last - gin->x_first, sector[i], row[i], pad[i], tim[i], theta);
        xyz[3 * i] = p.x; xyz[3 * i + 1] = p.y; xyz[3 * i + 2] = p.z;
    }
    return 0;
}

/* S8 on exact points: hits (sector, x, y, z) in hit order, used as both measurements and seed.
 * With ref (8 values, may be NULL) the reference measurements at the vertex are added (kf_anchor)
 * and the state is reported at x = 0. */
int or_fit_xyz(const or_geom_in *gin, int32_t nh, const int32_t *sector, const double *xyz, double *par,
               double *xref, double *cov, double *chi2, const double *ref) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    if (nh < 3 || nh > OR_MAX_ROWS * 4) return 0;
    int ks[OR_MAX_ROWS * 4];
    or_pt m[OR_MAX_ROWS * 4];
    for (int i = 0; i < nh; i++) {
        ks[i] = sector[i];
        m[i].x = xyz[3 * i];
        m[i].y = xyz[3 * i + 1];
        m[i].z = xyz[3 * i + 2];
        m[i].jy = m[i].jz = 1.0;
    }
    or_kf s;
    int ok = fit_points(&g, nh, ks, m, &m[0], &m[(nh - 1) / 2], &m[nh - 1], 0, &s);
    if (ok && ref) ok = kf_anchor(&g, &s, ref);
    if (!ok) return 0;
    for (int i = 0; i < 5; i++) par[i] = s.p[i];
    int k = 0;
    for (int i = 0; i < 5; i++) for (int j = 0; j <= i; j++) cov[k++] = s.P[i][j];
    *xref = s.x;
    *chi2 = s.chi2;
    return 1;
}

/* One propagation step (state and Jacobian) for the closed-form and finite-difference pins. */
int or_propagate(const or_geom_in *gin, double x, const double *p, double xh, double *pout, double *F) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    double FF[5][5];
    if (!prop_step(&g, x, p, xh, pout, FF)) return 0;
    for (int i = 0; i < 5; i++) for (int j = 0; j < 5; j++) F[i * 5 + j] = FF[i][j];
    return 1;
}

/* S7 decision alone on integer end points (for the edge pins): 1 and *D on a match, else 0. */
int or_merge_decide(const or_geom_in *gin, int32_t ks, const int64_t *s_end, int32_t kt, const int64_t *t_first,
                    int64_t *D) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    *D = -1;
    return merge_decide(&g, ks, s_end[0], s_end[1], s_end[2], s_end[3], s_end[4], s_end[5], kt, t_first[0],
                        t_first[1], t_first[2], D);
}

/* ============================================================================================
 * TPC-ITS matching for the drift calibration (sections 2.1 and 6: the TPC drift is calibrated by
 * matching TPC tracks to the tracks of the inner tracker).  Reading: every fitted TPC track (state
 * and covariance at its first hit, in the frame of that hit's sector) is extrapolated by the exact
 * helix step to x = 0, the production vertex; an ITS track (global azimuth phi0 of the momentum, z0,
 * tan lambda, q/pT at the vertex, with their errors) is expressed in the same frame, y = 0, sin phi =
 * sin(phi0 - alpha_k).  The drift calibration is unknown when matching, so z is not compared
 * beyond a loose window; the match chi2 is over (y, sin phi, tan lambda, q/pT) with the sum of the
 * TPC covariance and the ITS errors (sigma_y = OR_ITS_SIGMA_Y at the vertex).  Candidates: azimuth
 * within OR_ITS_DPHI, tan lambda within OR_ITS_DTL, z within OR_ITS_DZ; chi2 <= OR_ITS_CHI2.  Each
 * side keeps its best partner by (floor(chi2 * 2^20), index); mutual best pairs are matched.
 * ========================================================================================== */
#define OR_ITS_SIGMA_Y 0.01
#define OR_ITS_DPHI    0.1
#define OR_ITS_DTL     0.1
#define OR_ITS_DZ      2.0
#define OR_ITS_CHI2    100.0

/* a - 2 pi n, n the nearest integer (IEEE remainder): the angle wrapped into [-pi, pi] */
static double wrap_pi(double a) { return remainder(a, 2.0 * OR_PI); }

/* chi2 = d^T A^-1 d for a symmetric positive definite 4x4 A (Cholesky); returns -1 if A is not */
static double chi2_4(double A[4][4], const double *d) {
    double L[4][4] = {{0}};
    for (int i = 0; i < 4; i++) {
        for (int j = 0; j <= i; j++) {
            double v = A[i][j];
            for (int k = 0; k < j; k++) v -= L[i][k] * L[j][k];
            if (i == j) {
                if (v <= 0.0) return -1.0;
                L[i][i] = sqrt(v);
            } else {
                L[i][j] = v / L[j][j];
            }
        }
    }
    double y[4];
    for (int i = 0; i < 4; i++) {
        double v = d[i];
        for (int k = 0; k < i; k++) v -= L[i][k] * y[k];
        y[i] = v / L[i][i];
    }
    return y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3];
}

int or_its_match(const or_geom_in *gin, int32_t n_trk, const double *par, const double *cov, const double *xref,
                 const int32_t *ndf, const int32_t *sector, int32_t n_its, const double *its, int32_t *match_trk,
                 int32_t *match_its, double *chi2_out) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    int64_t *bt = (int64_t *)malloc(sizeof(int64_t) * (n_trk + 1));
    int64_t *bi = (int64_t *)malloc(sizeof(int64_t) * (n_its + 1));
    double *bchi = (double *)malloc(sizeof(double) * (n_trk + 1));
    for (int32_t t = 0; t < n_trk; t++) { bt[t] = -1; match_trk[t] = -1; bchi[t] = 0.0; }
    for (int32_t i = 0; i < n_its; i++) { bi[i] = -1; match_its[i] = -1; }
    const int64_t SHIFT = (int64_t)1 << 32;
    for (int32_t t = 0; t < n_trk; t++) {
        if (ndf[t] <= 0) continue;
        or_kf s;
        memset(&s, 0, sizeof(s));
        s.x = xref[t];
        s.ok = 1;
        s.frame = sector[t];
        int m = 0;
        for (int i = 0; i < 5; i++) s.p[i] = par[t * 5 + i];
        for (int i = 0; i < 5; i++) for (int j = 0; j <= i; j++) { s.P[i][j] = s.P[j][i] = cov[t * 15 + m]; m++; }
        kf_propagate(&g, &s, 0.0);
        if (!s.ok) continue;
        const double alpha = ((sector[t] % (g.n_sectors / 2)) + 0.5) * 2.0 * g.half_angle;
        const double phi_t = alpha + asin(s.p[2]);
        const int ix[4] = {0, 2, 3, 4};
        for (int32_t i = 0; i < n_its; i++) {
            const double *r = its + 8 * (int64_t)i;
            if (fabs(wrap_pi(r[0] - phi_t)) > OR_ITS_DPHI) continue;
            if (fabs(r[2] - s.p[3]) > OR_ITS_DTL || fabs(r[1] - s.p[1]) > OR_ITS_DZ) continue;
            const double dphi = wrap_pi(r[0] - alpha);
            const double d[4] = {s.p[0], s.p[2] - sin(dphi), s.p[3] - r[2], s.p[4] - r[3]};
            const double ev[4] = {OR_ITS_SIGMA_Y * OR_ITS_SIGMA_Y, pow(cos(dphi) * r[4], 2), r[6] * r[6], r[7] * r[7]};
            double A[4][4];
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++) A[a][b] = s.P[ix[a]][ix[b]] + (a == b ? ev[a] : 0.0);
            const double c2 = chi2_4(A, d);
            if (c2 < 0.0 || c2 > OR_ITS_CHI2) continue;
            const int64_t q = (int64_t)floor(c2 * 1048576.0);
            const int64_t kt = q * SHIFT + i, ki = q * SHIFT + t;
            if (bt[t] < 0 || kt < bt[t]) { bt[t] = kt; bchi[t] = c2; }
            if (bi[i] < 0 || ki < bi[i]) bi[i] = ki;
        }
    }
    for (int32_t t = 0; t < n_trk; t++) {
        if (bt[t] < 0) continue;
        const int32_t i = (int32_t)(bt[t] % SHIFT);
        if (bi[i] >= 0 && (int32_t)(bi[i] % SHIFT) == t && bi[i] / SHIFT == bt[t] / SHIFT) {
            match_trk[t] = i;
            match_its[i] = t;
            if (chi2_out) chi2_out[t] = bchi[t];
        }
    }
    free(bt); free(bi); free(bchi);
    return 0;
}

int or_its_constants(double *out, int cap) {
    const double v[] = {OR_ITS_SIGMA_Y, OR_ITS_DPHI, OR_ITS_DTL, OR_ITS_DZ, OR_ITS_CHI2};
    int n = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < n && i < cap; i++) out[i] = v[i];
    return n;
}


/* ---- looper legs (reading of the segment merging of section 3 for low-pT loopers) ------------
 * A particle with 2R inside the TPC goes out to the point of its circle farthest from the beam and
 * comes back in: the tracker finds the two legs as two tracks, both fitted outwards in pad-row
 * order, so the returning leg's fit has the opposite curvature and tan lambda of the outgoing one
 * and the same circle.  Every fitted track with 1/|C| <= RMAX whose circle centre lies at least
 * CMIN from the beam is a candidate: its circle (centre in the global frame, radius) and the z it
 * reaches at the far point of the circle, carried along the fitted direction from its first hit
 * (z + tan lambda * R * the turning angle to that point).  Two candidates of one event with
 * opposite curvature are a pair when their centres are within DC, radii within DR, far-point z
 * within DZ and |tan lambda_a + tan lambda_b| <= DTL; D = dcentre^2 + dR^2 + dz^2, and mutual
 * best pairs by (floor(D 2^20), index) are joined.  The outgoing leg is the one whose |z| grows
 * outwards (tan lambda times the side sign larger; the lower index on a tie). */
#define OR_LOOP_RMAX  130.0
#define OR_LOOP_CMIN  40.0
#define OR_LOOP_DC    5.0
#define OR_LOOP_DR    5.0
#define OR_LOOP_DZ    8.0
#define OR_LOOP_DTL   0.05

typedef struct { double cx, cy, R, zap, tl, sgn; int ok, side; } or_loop;

static or_loop loop_circle(const or_geom *g, const double *p, double xref, int sector, int ndf) {
    or_loop L;
    memset(&L, 0, sizeof(L));
    if (ndf <= 0 || !(fabs(p[2]) < 1.0)) return L;
    const double C = g->kB * p[4];
    if (!(fabs(C) * OR_LOOP_RMAX >= 1.0)) return L;
    const double sp = p[2], cp = sqrt(1.0 - sp * sp);
    /* centre of curvature in the sector frame: the point 1/C to the left of the direction */
    const double lx = xref - sp / C, ly = p[0] + cp / C;
    const double alpha = ((sector % (g->n_sectors / 2)) + 0.5) * 2.0 * g->half_angle;
    const double ca = cos(alpha), sa = sin(alpha);
    L.cx = lx * ca - ly * sa;
    L.cy = lx * sa + ly * ca;
    const double rc = sqrt(L.cx * L.cx + L.cy * L.cy);
    if (!(rc >= OR_LOOP_CMIN)) return L;
    L.R = 1.0 / fabs(C);
    /* first hit and far point of the circle, global frame */
    const double hx = xref * ca - p[0] * sa, hy = xref * sa + p[0] * ca;
    const double fx = L.cx + L.R * L.cx / rc, fy = L.cy + L.R * L.cy / rc;
    const double a_h = atan2(hy - L.cy, hx - L.cx), a_f = atan2(fy - L.cy, fx - L.cx);
    double turn = (a_f - a_h) * (C > 0.0 ? 1.0 : -1.0);   /* turning angle along the fit direction */
    turn = fmod(turn, 2.0 * OR_PI);
    if (turn < 0.0) turn += 2.0 * OR_PI;
    L.zap = p[1] + p[3] * L.R * turn;
    L.tl = p[3];
    L.sgn = C > 0.0 ? 1.0 : -1.0;
    L.side = sector < g->n_sectors / 2 ? 1 : -1;
    L.ok = 1;
    return L;
}

int or_looper_pairs(const or_geom_in *gin, int32_t n_trk, const double *par, const double *xref,
                    const int32_t *ndf, const int32_t *sector, const int32_t *event, int32_t *pair, int32_t *leg,
                    double *D_out) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    or_loop *L = (or_loop *)malloc(sizeof(or_loop) * (n_trk + 1));
    int64_t *best = (int64_t *)malloc(sizeof(int64_t) * (n_trk + 1));
    double *bD = (double *)malloc(sizeof(double) * (n_trk + 1));
    const int64_t SHIFT = (int64_t)1 << 32;
    for (int32_t t = 0; t < n_trk; t++) {
        L[t] = loop_circle(&g, par + 5 * (int64_t)t, xref[t], sector[t], ndf[t]);
        best[t] = -1;
        bD[t] = 0.0;
        pair[t] = -1;
        if (leg) leg[t] = 0;
    }
    for (int32_t a = 0; a < n_trk; a++) {
        if (!L[a].ok) continue;
        for (int32_t b = 0; b < n_trk; b++) {
            if (b == a || !L[b].ok || event[b] != event[a] || L[b].sgn == L[a].sgn) continue;
            const double dx = L[a].cx - L[b].cx, dy = L[a].cy - L[b].cy;
            const double dc2 = dx * dx + dy * dy, dR = L[a].R - L[b].R, dz = L[a].zap - L[b].zap;
            if (dc2 > OR_LOOP_DC * OR_LOOP_DC || fabs(dR) > OR_LOOP_DR || fabs(dz) > OR_LOOP_DZ) continue;
            if (fabs(L[a].tl + L[b].tl) > OR_LOOP_DTL) continue;
            const double D = dc2 + dR * dR + dz * dz;
            const int64_t k = (int64_t)floor(D * 1048576.0) * SHIFT + b;
            if (best[a] < 0 || k < best[a]) { best[a] = k; bD[a] = D; }
        }
    }
    for (int32_t a = 0; a < n_trk; a++) {
        if (best[a] < 0) continue;
        const int32_t b = (int32_t)(best[a] % SHIFT);
        if (best[b] < 0 || (int32_t)(best[b] % SHIFT) != a) continue;
        pair[a] = b;
        if (D_out) D_out[a] = bD[a];
        if (leg) {
            const double ua = L[a].tl * L[a].side, ub = L[b].tl * L[b].side;
            leg[a] = (ua > ub || (ua == ub && a < b)) ? 1 : 2;
        }
    }
    free(L); free(best); free(bD);
    return 0;
}

int or_loop_constants(double *out, int cap) {
    const double v[] = {OR_LOOP_RMAX, OR_LOOP_CMIN, OR_LOOP_DC, OR_LOOP_DR, OR_LOOP_DZ, OR_LOOP_DTL};
    int n = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < n && i < cap; i++) out[i] = v[i];
    return n;
}

/* The candidate description of one fitted track (test access): out = centre x, y (global), R,
 * far-point z, tan lambda, curvature sign; returns 1 for a candidate, 0 otherwise. */
int or_loop_circle(const or_geom_in *gin, const double *par, double xref, int32_t sector, int32_t ndf,
                   double *out) {
    or_geom g;
    if (make_geom(gin, &g)) return -1;
    const or_loop L = loop_circle(&g, par, xref, sector, ndf);
    out[0] = L.cx; out[1] = L.cy; out[2] = L.R; out[3] = L.zap; out[4] = L.tl; out[5] = L.sgn;
    return L.ok;
}
