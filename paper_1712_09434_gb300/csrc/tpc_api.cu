// Host side of the C ABI declared in include/tpc.h: context, workspace, argument validation,
// the per-event pipeline, its CUDA-graph replay for batches, and the refit/adjoint call.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "tpc_common.cuh"

using namespace tpc;

struct tpc_ctx {
    int device;
    int sm_count;
    tpc_geometry geom;
    double bz;
    DevGeom hgeom;
    DevGeom *dgeom;
    float *theta0;            // nominal calibration (FP32, device)
    // reservation
    int max_clusters, max_events, nbins_max, cap_chains;
    void *arena;
    size_t arena_bytes;
    Work ws;                  // workspace part of the kernel arguments
    float *ck, *rec;
    double *part;
    int32_t *order, *lhist;   // tracks by decreasing length for the adjoint
    // batch graph cache
    cudaStream_t cap_stream;
    // a few graphs, keyed by the kernel arguments (e.g. double-buffered inputs), least recently
    // used replaced first
    static constexpr int kGraphs = 4;
    cudaGraphExec_t gexec[kGraphs];
    Work gwork[kGraphs];
    bool ghasref[kGraphs];        // the graph also holds the refit / adjoint of the tracks
    const double *gref_theta[kGraphs];
    const float *gref_weight[kGraphs], *gref_anchor[kGraphs];
    int32_t gref_model[kGraphs];
    double *gref_sum[kGraphs], *gref_grad[kGraphs];
    bool gvalid[kGraphs];
    int gprofile[kGraphs];
    long long gused[kGraphs];
    long long gclock;
    // per-stage timing (tpc_profile_*): events between the stages of the last call of each kind
    int profile;
    cudaEvent_t ev_pipe[TPC_N_PIPE_STAGES + 1];
    cudaEvent_t ev_refit[TPC_N_REFIT_STAGES + 1];
    bool pipe_pending, refit_pending;
    double acc_ms[TPC_N_PIPE_STAGES + TPC_N_REFIT_STAGES];
    int acc_calls;
    // launch shapes set by tpc_set_tuning (used when a call passes no tuning of its own)
    tpc_tuning tune;
    bool has_tune;
    int32_t rules;            // TPC_RULE_* bits set by tpc_set_rules
};

namespace {

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return TPC_OK;
    std::fprintf(stderr, "libtpc: CUDA error %s\n", cudaGetErrorString(e));
    return TPC_ERR_CUDA;
}

#define TPC_CUDA(x)                              \
    do {                                         \
        const int rc__ = cuda_err((x));          \
        if (rc__ != TPC_OK) return rc__;         \
    } while (0)

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

template <class P>
void carve(char *&cur, P *&ptr, size_t count) {
    ptr = reinterpret_cast<P *>(cur);
    cur += align_up(count * sizeof(P));
}

// Lay out (or size, if base == nullptr) the workspace for the reservation.
size_t layout(tpc_ctx *c, char *base) {
    char *cur = base;
    const size_t N = (size_t)c->max_clusters + 1;
    const size_t nb = (size_t)c->nbins_max + 1;
    const size_t npad = N + 8 * (nb + 2) + 64;
    const size_t C = (size_t)c->cap_chains + 1;
    Work &w = c->ws;
    carve(cur, w.bin_ok, nb + 1);
    carve(cur, w.gyz, npad);
    carve(cur, w.gloc, npad);
    carve(cur, w.zoff, nb * ZOFF_STRIDE);
    carve(cur, w.up, N);
    carve(cur, w.down, N);
    carve(cur, w.clen, N);
    carve(cur, w.bin_cnt, nb + 1);
    carve(cur, w.chain_off, nb + 1);
    carve(cur, w.chain_start, C);
    carve(cur, w.chain_len, C);
    carve(cur, w.chain_bin, C);
    carve(cur, w.cand_n, C);
    carve(cur, w.cand_rows, C);
    carve(cur, w.cand_slots, C * c->hgeom.n_rows);
    carve(cur, w.claim, 2 * N);
    carve(cur, w.owner, N);
    carve(cur, w.cstate, C);
    carve(cur, w.seg_n, C);
    carve(cur, w.bestT, C);
    carve(cur, w.bestS, C);
    carve(cur, w.next, C);
    carve(cur, w.prev, C);
    carve(cur, w.inend, C);
    carve(cur, w.mrg_off, nb + 1);
    carve(cur, w.mrg_list, C);
    carve(cur, w.outend, 2 * C);
    carve(cur, w.sec_ymax, (size_t)c->max_events * c->hgeom.n_sectors + 1);
    carve(cur, w.head, C);
    carve(cur, w.head_id, C + 1);
    carve(cur, w.trk_n, C + 1);
    carve(cur, w.trk_head, C);
    carve(cur, w.trk_pack, 2 * N);
    carve(cur, w.gap_state, 6 * C);
    carve(cur, w.gap_bestT, C);
    carve(cur, w.gap_bestS, C);
    size_t scan_n = N > C ? N : C;
    scan_n = scan_n > nb ? scan_n : nb;
    const size_t scan_len = (size_t)scan_tmp_needed((int)scan_n) + 16;
    carve(cur, w.scan_tmp, scan_len);
    w.scan_tmp_len = (int)scan_len;
    carve(cur, w.counters, 64);
    carve(cur, w.status, 8);
    carve(cur, c->ck, refit_ck_words((long long)N, (long long)C));
    carve(cur, c->rec, (size_t)refit_rec_words((int)C));
    carve(cur, c->part, (size_t)refit_part_doubles((int)C, c->hgeom.n_sectors));
    carve(cur, c->order, C + 1);
    carve(cur, c->lhist, 1024);
    w.cap_chains = c->cap_chains;
    return (size_t)(cur - base);
}

int validate_in(const tpc_ctx *c, const tpc_clusters *in) {
    if (!in || !in->bin_off || in->n_events < 1 || in->n_clusters < 0) return TPC_ERR_INVALID_ARG;
    if (in->n_clusters > 0 && (!in->pad_fp || !in->time_fp)) return TPC_ERR_INVALID_ARG;
    if (c->arena == nullptr || in->n_clusters > c->max_clusters || in->n_events > c->max_events)
        return TPC_ERR_NOT_RESERVED;
    return TPC_OK;
}

int validate_out(const tpc_tracks *o) {
    if (!o || !o->label || !o->trk_off || !o->trk_hits || !o->ev_trk_off || !o->par || !o->xref || !o->cov ||
        !o->chi2 || !o->ndf || !o->n_tracks || o->cap_tracks < 1 || o->cap_hits < 1)
        return TPC_ERR_INVALID_ARG;
    return TPC_OK;
}

// largest block size each tunable kernel is compiled for (__launch_bounds__)
const int kMaxBlock[TPC_N_TUNE] = {256, 128, 256, 128, 1024, 512, 128, 128};

Work make_work(const tpc_ctx *c, const tpc_clusters *in, const tpc_tracks *o, const tpc_tuning *tune) {
    Work w = c->ws;
    w.pad = in->pad_fp;
    w.tim = in->time_fp;
    w.bin_off_in = in->bin_off;
    w.bin_off = w.bin_ok;
    w.n_events = in->n_events;
    w.n_clusters = in->n_clusters;
    w.nbins = in->n_events * c->hgeom.n_sectors * c->hgeom.n_rows;
    w.ns = c->hgeom.n_sectors;
    w.nr = c->hgeom.n_rows;
    w.rules = c->rules;
    w.geom = c->dgeom;
    w.sm_count = c->sm_count;
    w.label = o->label;
    w.trk_off = o->trk_off;
    w.trk_hits = o->trk_hits;
    w.ev_trk_off = o->ev_trk_off;
    w.par = o->par;
    w.xref = o->xref;
    w.cov = o->cov;
    w.chi2 = o->chi2;
    w.ndf = o->ndf;
    w.n_tracks = o->n_tracks;
    // tracks <= accepted segments <= cap_chains and hits <= clusters: larger capacities are clamped
    w.cap_tracks = o->cap_tracks < c->cap_chains ? o->cap_tracks : c->cap_chains;
    w.cap_hits = o->cap_hits < c->max_clusters + 1 ? o->cap_hits : c->max_clusters + 1;
    std::memset(&w.tune, 0, sizeof(w.tune));
    if (!tune && c->has_tune) tune = &c->tune;
    if (tune) {
        for (int k = 0; k < TPC_N_TUNE; k++) {
            w.tune.block[k] = tune->block[k] > 0 && tune->block[k] % 32 == 0 && tune->block[k] <= kMaxBlock[k] ? tune->block[k] : 0;
            w.tune.grid[k] = tune->ctas_per_sm[k] > 0 ? tune->ctas_per_sm[k] * c->sm_count : 0;
            w.tune.chunk[k] = tune->chunk[k] > 0 ? tune->chunk[k] : 0;
        }
    }
    return w;
}

// The whole tracking path for the events in W, enqueued on s (no host synchronisation).  With
// profiling on, an event is recorded before the first and after every stage.
int enqueue_pipeline(const tpc_ctx *c, const Work &W, cudaStream_t s, bool capturing) {
    const bool prof = c->profile != 0;
    // inside a stream capture the records must become external event nodes of the graph
    const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_pipe[0], s, evf));
    TPC_CUDA(cudaMemsetAsync(W.counters, 0, 64 * sizeof(int32_t), s));
    if (W.n_clusters > 0) TPC_CUDA(cudaMemsetAsync(W.label, 0xff, (size_t)W.n_clusters * sizeof(int32_t), s));
    launch_bins_check(W, s);
    launch_grid(W, s);
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_pipe[1], s, evf));
    launch_links(W, s);
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_pipe[2], s, evf));
    launch_chains(W, s);
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_pipe[3], s, evf));
    launch_follow(W, s);
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_pipe[4], s, evf));
    launch_select(W, s);
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_pipe[5], s, evf));
    launch_merge(W, s);
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_pipe[6], s, evf));
    launch_len_order(W, c->order, c->lhist, s);
    launch_refit(W, c->theta0, c->order, s);
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_pipe[7], s, evf));
    return cuda_err(cudaGetLastError());
}

// Arguments of the refit / adjoint part of a whole-step graph.
struct RefitArgs {
    const double *theta;
    const float *weight, *anchor;
    int32_t model;
    double *sum, *grad;
};

// Refit under theta and its adjoint for the tracks counted in *n_tracks_dev (S0, S8, S9), enqueued
// on s.  With profiling on, events between the refit stages (external event nodes when capturing).
// pack = false when the tracking part of the same stream order has just checked the bin offsets
// and written the packed hits and the length order of exactly these tracks (the whole step as one
// graph).
int enqueue_refit_grad(const tpc_ctx *c, const Work &W, const int32_t *n_tracks_dev, const double *theta,
                       const float *weight, const float *anchor, int model, double *sum_chi2, double *grad,
                       cudaStream_t s, bool capturing, bool pack = true) {
    const bool prof = c->profile != 0;
    const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_refit[0], s, evf));
    // the refit reads the track count from the workspace counters
    TPC_CUDA(cudaMemcpyAsync(W.counters + CNT_NTRACKS, n_tracks_dev, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (pack) {
        TPC_CUDA(cudaMemsetAsync(W.counters + CNT_BINS_BAD, 0, sizeof(int32_t), s));
        launch_bins_check(W, s);
        launch_pack_hits(W, s);
    }
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_refit[1], s, evf));
    launch_refit_grad_fit(W, theta, weight, anchor, model, grad != nullptr, c->ck, (long long)c->max_clusters + 1,
                          (long long)c->cap_chains + 1, c->rec, c->order, c->lhist, !pack, s);
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_refit[2], s, evf));
    launch_refit_grad_reduce(W, sum_chi2, grad, c->rec, c->part, s);
    if (prof) TPC_CUDA(cudaEventRecordWithFlags(c->ev_refit[3], s, evf));
    return cuda_err(cudaGetLastError());
}

// The tracking pipeline (and, with ra, the refit / adjoint of its tracks) as one CUDA graph,
// captured once per argument set and replayed; a few graphs are cached, least recently used first
// out, and a recapture updates the executable graph in place when it can.
int launch_graph(tpc_ctx *c, const Work &W, const RefitArgs *ra, cudaStream_t s) {
    int slot = -1;
    for (int k = 0; k < tpc_ctx::kGraphs; k++) {
        if (!c->gvalid[k] || c->gprofile[k] != c->profile || c->ghasref[k] != (ra != nullptr) ||
            std::memcmp(&W, &c->gwork[k], sizeof(Work)) != 0)
            continue;
        if (ra && (c->gref_theta[k] != ra->theta || c->gref_weight[k] != ra->weight ||
                   c->gref_anchor[k] != ra->anchor || c->gref_model[k] != ra->model || c->gref_sum[k] != ra->sum ||
                   c->gref_grad[k] != ra->grad))
            continue;
        slot = k;
    }
    if (slot < 0) {
        slot = 0;   // an empty slot, else the least recently used
        for (int k = 0; k < tpc_ctx::kGraphs; k++) {
            if (!c->gvalid[k]) { slot = k; break; }
            if (c->gused[k] < c->gused[slot]) slot = k;
        }
        cudaGraph_t graph = nullptr;
        TPC_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        int erc = enqueue_pipeline(c, W, c->cap_stream, true);
        if (erc == TPC_OK && ra)
            erc = enqueue_refit_grad(c, W, W.n_tracks, ra->theta, ra->weight, ra->anchor, ra->model, ra->sum,
                                     ra->grad, c->cap_stream, true, false);
        const cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
        if (erc != TPC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return erc;
        }
        TPC_CUDA(ce);
        if (c->gvalid[slot]) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(c->gexec[slot], graph, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(c->gexec[slot]);
                c->gvalid[slot] = false;
            }
        }
        if (!c->gvalid[slot]) {
            const cudaError_t ie = cudaGraphInstantiate(&c->gexec[slot], graph, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(graph);
                return cuda_err(ie);
            }
        }
        cudaGraphDestroy(graph);
        c->gwork[slot] = W;
        c->ghasref[slot] = ra != nullptr;
        if (ra) {
            c->gref_theta[slot] = ra->theta;
            c->gref_weight[slot] = ra->weight;
            c->gref_anchor[slot] = ra->anchor;
            c->gref_model[slot] = ra->model;
            c->gref_sum[slot] = ra->sum;
            c->gref_grad[slot] = ra->grad;
        }
        c->gvalid[slot] = true;
        c->gprofile[slot] = c->profile;
    }
    c->gused[slot] = ++c->gclock;
    TPC_CUDA(cudaGraphLaunch(c->gexec[slot], s));
    return TPC_OK;
}

}  // namespace

extern "C" {

int tpc_init(const tpc_geometry *g, double bz_tesla, tpc_ctx **out) {
    if (!g || !out) return TPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (g->n_sectors < 2 || g->n_sectors % 2 || g->n_sectors > MAX_SECTORS || g->n_rows < 3 ||
        g->n_rows > MAX_ROWS || !(g->x_last > g->x_first) || !(g->x_first > 0) || !(g->lsb_cm > 0) ||
        !(g->z_max > 0) || !(g->half_angle_deg > 0) || g->z_max / g->lsb_cm > 65535.0 ||
        g->x_last * std::tan(g->half_angle_deg * M_PI / 180.0) / g->lsb_cm > 32767.0)
        return TPC_ERR_INVALID_ARG;
    tpc_ctx *c = new tpc_ctx();
    std::memset(c, 0, sizeof(*c));
    c->geom = *g;
    c->bz = bz_tesla;
    if (cuda_err(cudaGetDevice(&c->device)) ||
        cuda_err(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device))) {
        delete c;
        return TPC_ERR_CUDA;
    }
    DevGeom &h = c->hgeom;
    h.n_sectors = g->n_sectors;
    h.n_rows = g->n_rows;
    h.half = g->n_sectors / 2;
    const double ha = g->half_angle_deg * M_PI / 180.0;
    h.zmax = (int)std::llround(g->z_max / g->lsb_cm);
    h.c30 = std::llround(std::cos(2.0 * ha) * 1073741824.0);
    h.s30 = std::llround(std::sin(2.0 * ha) * 1073741824.0);
    h.kB = (float)(-0.299792458e-2 * bz_tesla);
    h.lsb = (float)g->lsb_cm;
    h.z_max = (float)g->z_max;
    h.x_first = (float)g->x_first;
    h.inv_span = (float)(1.0 / (g->x_last - g->x_first));
    h.pitch = (float)((g->x_last - g->x_first) / (g->n_rows - 1));
    for (int r = 0; r < g->n_rows; r++) {
        const double x = g->x_first + r * (g->x_last - g->x_first) / (g->n_rows - 1);
        h.xr[r] = (float)x;
        h.ymax[r] = (int)std::floor(x * std::tan(ha) / g->lsb_cm);
        h.xtab[r] = (int)std::llround(x / g->lsb_cm);
    }
    for (int m = -h.half; m <= h.half; m++) {
        h.rot_cos[m + h.half] = (float)std::cos(m * 2.0 * ha);
        h.rot_sin[m + h.half] = (float)std::sin(m * 2.0 * ha);
    }
    float th0[1 + 2 * MAX_SECTORS] = {0.f};
    th0[0] = 1.f;
    if (cuda_err(cudaMalloc(&c->dgeom, sizeof(DevGeom))) ||
        cuda_err(cudaMemcpy(c->dgeom, &h, sizeof(DevGeom), cudaMemcpyHostToDevice)) ||
        cuda_err(cudaMalloc(&c->theta0, sizeof(th0))) ||
        cuda_err(cudaMemcpy(c->theta0, th0, sizeof(th0), cudaMemcpyHostToDevice)) ||
        cuda_err(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking))) {
        tpc_destroy(c);
        return TPC_ERR_CUDA;
    }
    prepare_kernels();
    *out = c;
    return TPC_OK;
}

int tpc_reserve(tpc_ctx *c, int32_t max_clusters, int32_t max_events) {
    if (!c || max_clusters < 0 || max_events < 1) return TPC_ERR_INVALID_ARG;
    if (c->arena && max_clusters <= c->max_clusters && max_events <= c->max_events) return TPC_OK;
    const long long nbins = (long long)max_events * c->hgeom.n_sectors * c->hgeom.n_rows;
    if (nbins > (1ll << 30)) return TPC_ERR_INVALID_ARG;
    if (c->arena) {
        TPC_CUDA(cudaDeviceSynchronize());
        cudaFree(c->arena);
        c->arena = nullptr;
    }
    for (int k = 0; k < tpc_ctx::kGraphs; k++)
        if (c->gvalid[k]) {
            cudaGraphExecDestroy(c->gexec[k]);
            c->gvalid[k] = false;
        }
    c->max_clusters = max_clusters > c->max_clusters ? max_clusters : c->max_clusters;
    c->max_events = max_events > c->max_events ? max_events : c->max_events;
    c->nbins_max = c->max_events * c->hgeom.n_sectors * c->hgeom.n_rows;
    c->cap_chains = c->max_clusters / N_SEED + 1;
    const size_t bytes = layout(c, nullptr) + 4096;
    void *p = nullptr;
    TPC_CUDA(cudaMalloc(&p, bytes));
    c->arena = p;
    c->arena_bytes = bytes;
    layout(c, static_cast<char *>(p));
    TPC_CUDA(cudaMemset(c->ws.status, 0, 8 * sizeof(int32_t)));
    return TPC_OK;
}

void tpc_destroy(tpc_ctx *c) {
    if (!c) return;
    for (auto &e : c->ev_pipe) if (e) cudaEventDestroy(e);
    for (auto &e : c->ev_refit) if (e) cudaEventDestroy(e);
    for (int k = 0; k < tpc_ctx::kGraphs; k++)
        if (c->gvalid[k]) cudaGraphExecDestroy(c->gexec[k]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->arena) cudaFree(c->arena);
    if (c->dgeom) cudaFree(c->dgeom);
    if (c->theta0) cudaFree(c->theta0);
    delete c;
}

int tpc_set_tuning(tpc_ctx *c, const tpc_tuning *tune) {
    if (!c) return TPC_ERR_INVALID_ARG;
    if (tune) {
        for (int k = 0; k < TPC_N_TUNE; k++)
            if (tune->block[k] < 0 || tune->ctas_per_sm[k] < 0 || tune->chunk[k] < 0 ||
                (tune->block[k] > 0 && (tune->block[k] % 32 != 0 || tune->block[k] > kMaxBlock[k])) ||
                tune->ctas_per_sm[k] > 64 || tune->chunk[k] > 64)
                return TPC_ERR_INVALID_ARG;
        c->tune = *tune;
        c->has_tune = true;
    } else {
        c->has_tune = false;
    }
    return TPC_OK;
}

int tpc_track_event(tpc_ctx *c, const tpc_clusters *in, tpc_tracks *out, void *stream) {
    if (!c) return TPC_ERR_INVALID_ARG;
    int rc = validate_in(c, in);
    if (rc) return rc;
    if ((rc = validate_out(out))) return rc;
    const Work W = make_work(c, in, out, nullptr);
    rc = enqueue_pipeline(c, W, static_cast<cudaStream_t>(stream), false);
    if (rc == TPC_OK && c->profile) c->pipe_pending = true;
    return rc;
}

int tpc_track_batch(tpc_ctx *c, const tpc_clusters *in, tpc_tracks *out, const tpc_tuning *tune, void *stream) {
    if (!c) return TPC_ERR_INVALID_ARG;
    int rc = validate_in(c, in);
    if (rc) return rc;
    if ((rc = validate_out(out))) return rc;
    const Work W = make_work(c, in, out, tune);
    rc = launch_graph(c, W, nullptr, static_cast<cudaStream_t>(stream));
    if (rc == TPC_OK && c->profile) c->pipe_pending = true;
    return rc;
}

int tpc_refit_grad(tpc_ctx *c, const tpc_clusters *in, const tpc_tracks *trk, const double *theta,
                   const float *weight, const float *anchor, int32_t error_model, double *sum_chi2, double *grad,
                   void *stream) {
    if (!c || !theta || !sum_chi2 || !trk || !trk->trk_off || !trk->trk_hits || !trk->n_tracks ||
        trk->cap_tracks < 1)
        return TPC_ERR_INVALID_ARG;
    if (anchor && (reinterpret_cast<uintptr_t>(anchor) & 15u)) return TPC_ERR_INVALID_ARG;
    if (error_model != TPC_ERRORS_FIXED && error_model != TPC_ERRORS_RAW) return TPC_ERR_INVALID_ARG;
    int rc = validate_in(c, in);
    if (rc) return rc;
    const Work W = make_work(c, in, trk, nullptr);
    rc = enqueue_refit_grad(c, W, trk->n_tracks, theta, weight, anchor, error_model, sum_chi2, grad,
                            static_cast<cudaStream_t>(stream), false);
    if (rc == TPC_OK && c->profile) c->refit_pending = true;
    return rc;
}

int tpc_track_refit_batch(tpc_ctx *c, const tpc_clusters *in, tpc_tracks *out, const double *theta,
                          const float *weight, const float *anchor, int32_t error_model, double *sum_chi2,
                          double *grad, const tpc_tuning *tune, void *stream) {
    if (!c || !theta || !sum_chi2) return TPC_ERR_INVALID_ARG;
    if (anchor && (reinterpret_cast<uintptr_t>(anchor) & 15u)) return TPC_ERR_INVALID_ARG;
    if (error_model != TPC_ERRORS_FIXED && error_model != TPC_ERRORS_RAW) return TPC_ERR_INVALID_ARG;
    int rc = validate_in(c, in);
    if (rc) return rc;
    if ((rc = validate_out(out))) return rc;
    const Work W = make_work(c, in, out, tune);
    const RefitArgs ra{theta, weight, anchor, error_model, sum_chi2, grad};
    rc = launch_graph(c, W, &ra, static_cast<cudaStream_t>(stream));
    if (rc == TPC_OK && c->profile) c->pipe_pending = c->refit_pending = true;
    return rc;
}

int tpc_its_match(tpc_ctx *c, const tpc_clusters *in, const tpc_tracks *trk, const float *its, int32_t n_its,
                  int32_t *match_trk, int32_t *match_its, float *anchor, void *stream) {
    if (!c || !trk || !trk->trk_off || !trk->trk_hits || !trk->par || !trk->cov || !trk->xref || !trk->ndf ||
        !trk->n_tracks || trk->cap_tracks < 1 || !match_trk || n_its < 0 || (n_its > 0 && (!its || !match_its)))
        return TPC_ERR_INVALID_ARG;
    if (anchor && (reinterpret_cast<uintptr_t>(anchor) & 15u)) return TPC_ERR_INVALID_ARG;
    int rc = validate_in(c, in);
    if (rc) return rc;
    if (n_its > c->cap_chains || its_match_nphi() > c->nbins_max) return TPC_ERR_CAPACITY;
    const Work W = make_work(c, in, trk, nullptr);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TPC_CUDA(cudaMemsetAsync(W.counters + CNT_BINS_BAD, 0, sizeof(int32_t), s));
    launch_bins_check(W, s);
    const double ha = c->geom.half_angle_deg * M_PI / 180.0;
    launch_its_match(W, its, n_its, match_trk, match_its, anchor, -0.299792458e-2 * c->bz, ha, 2.0 * ha, s);
    return cuda_err(cudaGetLastError());
}

int tpc_looper_pairs(tpc_ctx *c, const tpc_clusters *in, const tpc_tracks *trk, int32_t *pair, int32_t *leg,
                     void *stream) {
    if (!c || !trk || !trk->trk_off || !trk->trk_hits || !trk->par || !trk->xref || !trk->ndf || !trk->n_tracks ||
        trk->cap_tracks < 1 || !pair)
        return TPC_ERR_INVALID_ARG;
    int rc = validate_in(c, in);
    if (rc) return rc;
    if ((long long)in->n_events * loop_nphi() > c->nbins_max) return TPC_ERR_CAPACITY;
    const Work W = make_work(c, in, trk, nullptr);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TPC_CUDA(cudaMemsetAsync(W.counters + CNT_BINS_BAD, 0, sizeof(int32_t), s));
    launch_bins_check(W, s);
    // candidate records (8 doubles and 8 floats per track) in the refit workspace, free between calls
    const long long rec_tracks = (long long)refit_ck_words((long long)c->max_clusters + 1, (long long)c->cap_chains + 1) / 24;
    const int nt_cap = (int)std::min<long long>(c->cap_chains, rec_tracks);
    const double ha = c->geom.half_angle_deg * M_PI / 180.0;
    launch_looper_pairs(W, pair, leg, -0.299792458e-2 * c->bz, ha, 2.0 * ha, reinterpret_cast<double *>(c->ck),
                        nt_cap, s);
    return cuda_err(cudaGetLastError());
}

int tpc_merge_slices(tpc_ctx *c, const tpc_clusters *in, const tpc_tracks *slice_trk, int32_t slice_len,
                     tpc_tracks *frame, void *stream) {
    if (!c) return TPC_ERR_INVALID_ARG;
    int rc = validate_in(c, in);
    if (rc) return rc;
    if (!slice_trk || !slice_trk->trk_off || !slice_trk->trk_hits || !slice_trk->ev_trk_off || !slice_trk->n_tracks)
        return TPC_ERR_INVALID_ARG;
    if (!frame || !frame->label || !frame->trk_off || !frame->trk_hits || !frame->n_tracks || frame->cap_tracks < 1 ||
        frame->cap_hits < 1)
        return TPC_ERR_INVALID_ARG;
    if (slice_len < 1 || slice_len > c->hgeom.zmax + 1) return TPC_ERR_INVALID_ARG;
    Work W = make_work(c, in, frame, nullptr);
    W.s_trk_off = slice_trk->trk_off;
    W.s_trk_hits = slice_trk->trk_hits;
    W.s_ev_trk_off = slice_trk->ev_trk_off;
    W.s_n_tracks = slice_trk->n_tracks;
    W.slice_len = slice_len;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TPC_CUDA(cudaMemsetAsync(W.counters + CNT_BINS_BAD, 0, sizeof(int32_t), s));
    launch_bins_check(W, s);
    launch_frame_merge(W, s);
    return cuda_err(cudaGetLastError());
}

int tpc_profile_enable(tpc_ctx *c, int enable) {
    if (!c) return TPC_ERR_INVALID_ARG;
    if (enable && !c->ev_pipe[0]) {
        for (auto &e : c->ev_pipe) TPC_CUDA(cudaEventCreate(&e));
        for (auto &e : c->ev_refit) TPC_CUDA(cudaEventCreate(&e));
    }
    c->profile = enable ? 1 : 0;
    return TPC_OK;
}

int tpc_profile_read(tpc_ctx *c, double *ms, int32_t cap, int32_t *n_calls) {
    if (!c || !ms) return TPC_ERR_INVALID_ARG;
    if (c->pipe_pending) {
        TPC_CUDA(cudaEventSynchronize(c->ev_pipe[TPC_N_PIPE_STAGES]));
        for (int i = 0; i < TPC_N_PIPE_STAGES; i++) {
            float t = 0.f;
            TPC_CUDA(cudaEventElapsedTime(&t, c->ev_pipe[i], c->ev_pipe[i + 1]));
            c->acc_ms[i] += t;
        }
        c->pipe_pending = false;
        c->acc_calls++;
    }
    if (c->refit_pending) {
        TPC_CUDA(cudaEventSynchronize(c->ev_refit[TPC_N_REFIT_STAGES]));
        for (int i = 0; i < TPC_N_REFIT_STAGES; i++) {
            float t = 0.f;
            TPC_CUDA(cudaEventElapsedTime(&t, c->ev_refit[i], c->ev_refit[i + 1]));
            c->acc_ms[TPC_N_PIPE_STAGES + i] += t;
        }
        c->refit_pending = false;
    }
    const int n = TPC_N_PIPE_STAGES + TPC_N_REFIT_STAGES;
    for (int i = 0; i < n && i < cap; i++) ms[i] = c->acc_ms[i];
    if (n_calls) *n_calls = c->acc_calls;
    if (cap < 0) {   /* reset */
        for (int i = 0; i < n; i++) c->acc_ms[i] = 0.0;
        c->acc_calls = 0;
    }
    return n;
}

int tpc_set_rules(tpc_ctx *c, int32_t rules) {
    if (!c || (rules & ~(TPC_RULE_SKIP_ROW | TPC_RULE_GAP_MERGE))) return TPC_ERR_INVALID_ARG;
    c->rules = rules;
    return TPC_OK;
}

int tpc_match_constants(double *out, int32_t cap) {
    double v[16];
    int n = its_constants(v);
    n += loop_constants(v + n);
    if (out)
        for (int i = 0; i < n && i < cap; i++) out[i] = v[i];
    return n;
}

int tpc_rule_constants(int64_t *out, int32_t cap) {
    const int64_t v[] = {TPC_RULE_SKIP_ROW, TPC_RULE_GAP_MERGE, GAP_MAX};
    const int n = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < n && i < cap; i++) out[i] = v[i];
    return n;
}

int tpc_sync_status(tpc_ctx *c, void *stream) {
    if (!c || !c->arena) return TPC_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TPC_CUDA(cudaStreamSynchronize(s));
    int32_t st = 0;
    TPC_CUDA(cudaMemcpy(&st, c->ws.status, sizeof(st), cudaMemcpyDeviceToHost));
    TPC_CUDA(cudaMemset(c->ws.status, 0, sizeof(int32_t)));
    if (st & ST_TIMEOUT) return TPC_ERR_TIMEOUT;
    if (st & ST_BOUNDS) return TPC_ERR_BOUNDS;
    if (st & ST_CAPACITY) return TPC_ERR_CAPACITY;
    return TPC_OK;
}

const char *tpc_strerror(int code) {
    switch (code) {
        case TPC_OK: return "ok";
        case TPC_ERR_INVALID_ARG: return "invalid argument";
        case TPC_ERR_CAPACITY: return "output or workspace capacity too small";
        case TPC_ERR_TIMEOUT: return "bounded device wait or iteration limit exceeded";
        case TPC_ERR_CUDA: return "CUDA runtime error";
        case TPC_ERR_BOUNDS: return "input index or coordinate out of range";
        case TPC_ERR_NOT_RESERVED: return "workspace smaller than the call (tpc_reserve)";
        default: return "unknown error";
    }
}

int tpc_debug_copy(tpc_ctx *c, int32_t what, void *dst, int64_t dst_bytes, void *stream) {
    if (!c || !c->arena || !dst) return TPC_ERR_INVALID_ARG;
    const Work &w = c->ws;
    const size_t N = (size_t)c->max_clusters, C = (size_t)c->cap_chains;
    const void *src = nullptr;
    size_t bytes = 0;
    switch (what) {
        case 0: src = w.up; bytes = N * 4; break;
        case 1: src = w.down; bytes = N * 4; break;
        case 2: src = w.counters + CNT_NCHAINS; bytes = 4; break;
        case 3: src = w.chain_start; bytes = C * 4; break;
        case 4: src = w.chain_len; bytes = C * 4; break;
        case 5: src = w.cand_n; bytes = C * 4; break;
        case 6: src = w.cand_slots; bytes = C * c->hgeom.n_rows * 4; break;
        case 7: src = w.cand_rows; bytes = C * 4; break;
        case 8: src = w.seg_n; bytes = C * 4; break;
        case 9: src = w.next; bytes = C * 4; break;
        case 10: src = w.counters; bytes = 16 * 4; break;
        case 11: src = c->rec; bytes = (size_t)refit_rec_words((int)(C + 1)) * 4; break;
        default: return TPC_ERR_INVALID_ARG;
    }
    if (dst_bytes < 0) return TPC_ERR_INVALID_ARG;
    if ((size_t)dst_bytes < bytes) bytes = (size_t)dst_bytes;
    TPC_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
    return TPC_OK;
}

int tpc_constants(int64_t *out, int32_t cap) {
    const int64_t v[] = {W_LINK, D_MAX, N_SEED, M_MISS, W_F0, W_F1, V_MAX, N_MIN, W_MERGE, MERGE_XMAX, MERGE_BACK};
    const int n = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < n && i < cap; i++) out[i] = v[i];
    return n;
}

}  // extern "C"
