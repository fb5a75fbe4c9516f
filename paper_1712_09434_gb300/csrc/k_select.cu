// S6 track selection: the exact result of the sequential greedy rule, computed in parallel rounds.
//
// Sequential rule: candidates in priority order (more hits first, then earlier seed) keep the hits
// that no already-accepted candidate owns and are accepted with at least N_MIN kept hits.  Hits
// belong to one sector, so one CTA handles one (event, sector) from a work queue.  Priority key
// (unique, smaller = earlier): ((n_rows - n_hits) << 23) | (candidate index in the sector).
//
// Round: every undecided candidate claims its hits (atomicMax on (round << 32 | ~key), so the
// latest round wins and inside it the smallest key); an undecided candidate whose hits are all
// resolved (owned by an accepted candidate = lost, or claimed by itself = kept) decides, and if
// accepted takes ownership of its kept hits at once; one that cannot reach N_MIN even with its
// unresolved hits is rejected.  The highest-priority undecided candidate always decides, so the
// rounds end, and every decision equals the sequential one (a candidate decides only when no
// higher-priority undecided candidate shares a hit with it).  Two barrier-separated phases per
// round; each lane loads its row slots first and their owner and claim words together.
#include "tpc_common.cuh"

namespace tpc {

namespace {

enum { CS_UNDECIDED = 0, CS_ACCEPTED = 2, CS_REJECTED = 3 };

constexpr int SEL_ILP = 5;   // row slots per lane loaded before their dependent loads (5 x 32 >= 159)

__device__ __forceinline__ uint32_t key_of(int n_rows, int n_hits, int local) {
    return ((uint32_t)(n_rows - n_hits) << 23) | (uint32_t)local;
}

// One warp per candidate inside each phase: the lanes walk the candidate's row slots 32 at a time
// (coalesced), so claims, counts and ownership of a ~100-hit candidate take a few warp steps.
__global__ void __launch_bounds__(1024) k_select(Work W) {
    __shared__ int s_item, s_undecided;
    const DevGeom &g = *W.geom;
    const int nr = g.n_rows, ns = g.n_sectors;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int n_chains = W.counters[CNT_NCHAINS];
    if (n_chains > W.cap_chains) n_chains = W.cap_chains;
    const int n_items = W.n_events * ns;
    int32_t *q = W.counters + CNT_Q0 + 4;
    unsigned long long *claim = reinterpret_cast<unsigned long long *>(W.claim);
    for (int it = queue_next(q, 1, &s_item); it < n_items; it = queue_next(q, 1, &s_item)) {
        const int b0 = it * nr;   // (event*ns + sector)*nr
        const int t0 = min(W.chain_off[b0], n_chains), t1 = min(W.chain_off[b0 + nr], n_chains);
        const int cl0 = W.bin_off[b0], cl1 = W.bin_off[b0 + nr];
        for (int c = cl0 + threadIdx.x; c < cl1; c += blockDim.x) {
            W.owner[c] = KEY_NONE;
            claim[c] = 0ull;
        }
        // a candidate with fewer than N_MIN hits can never be accepted: it is rejected up front
        // and never claims (the sequential rule gives it nothing either)
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x)
            W.cstate[t] = W.cand_n[t] < N_MIN ? CS_REJECTED : CS_UNDECIDED;
        __syncthreads();
        // Round k: the undecided candidates claim their unowned hits; then each decides.  A
        // candidate accepted in round k takes ownership of its kept hits at once: only the claimant
        // of a hit in round k can own it, and a later reader that already sees the owner counts
        // the hit as lost, which is the sequential answer for it (its owner is accepted).
        int round = 1;
        bool more = true;
        for (; more && round <= SELECT_MAX_ROUNDS; round++) {
            for (int t = t0 + warp; t < t1; t += nwarps) {
                if (W.cstate[t] != CS_UNDECIDED) continue;
                const uint32_t key = key_of(nr, W.cand_n[t], t - t0);
                const unsigned long long v = ((unsigned long long)round << 32) | (uint32_t)~key;
                const int rr = W.cand_rows[t];
                const int ra = rr & 0xffff, rb = rr >> 16;
                const int32_t *sl = W.cand_slots + (size_t)t * nr;
                for (int r0 = ra; r0 <= rb; r0 += 32 * SEL_ILP) {
                    int h[SEL_ILP];
#pragma unroll
                    for (int j = 0; j < SEL_ILP; j++) {
                        const int r = r0 + lane + 32 * j;
                        h[j] = r <= rb ? sl[r] : -1;
                    }
#pragma unroll
                    for (int j = 0; j < SEL_ILP; j++)
                        if (h[j] >= 0) atomicMax(claim + h[j], v);
                }
            }
            if (threadIdx.x == 0) s_undecided = 0;
            __syncthreads();
            for (int t = t0 + warp; t < t1; t += nwarps) {
                if (W.cstate[t] != CS_UNDECIDED) continue;
                const uint32_t key = key_of(nr, W.cand_n[t], t - t0);
                const unsigned long long v = ((unsigned long long)round << 32) | (uint32_t)~key;
                const int rr = W.cand_rows[t];
                const int ra = rr & 0xffff, rb = rr >> 16;
                const int32_t *sl = W.cand_slots + (size_t)t * nr;
                int sure = 0, unk = 0;
                int h[SEL_ILP];
                bool mine[SEL_ILP];
                for (int r0 = ra; r0 <= rb; r0 += 32 * SEL_ILP) {
                    unsigned long long cv[SEL_ILP];
                    uint32_t ov[SEL_ILP];
#pragma unroll
                    for (int j = 0; j < SEL_ILP; j++) {
                        const int r = r0 + lane + 32 * j;
                        h[j] = r <= rb ? sl[r] : -1;
                    }
#pragma unroll
                    for (int j = 0; j < SEL_ILP; j++)
                        if (h[j] >= 0) { ov[j] = W.owner[h[j]]; cv[j] = claim[h[j]]; }
#pragma unroll
                    for (int j = 0; j < SEL_ILP; j++) {
                        mine[j] = false;
                        if (h[j] < 0 || ov[j] != KEY_NONE) continue;       // miss, or lost
                        if (cv[j] == v) { sure++; mine[j] = true; } else { unk++; }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sure += __shfl_xor_sync(0xffffffffu, sure, o);
                    unk += __shfl_xor_sync(0xffffffffu, unk, o);
                }
                if (unk == 0 && sure >= N_MIN) {
                    if (rb - ra < 32 * SEL_ILP) {      // one pass: this lane's hits are in registers
#pragma unroll
                        for (int j = 0; j < SEL_ILP; j++)
                            if (mine[j]) W.owner[h[j]] = key;
                    } else {
                        for (int r = ra + lane; r <= rb; r += 32) {
                            const int hh = sl[r];
                            if (hh >= 0 && W.owner[hh] == KEY_NONE && claim[hh] == v) W.owner[hh] = key;
                        }
                    }
                }
                if (lane == 0) {
                    if (unk == 0) {
                        const bool acc = sure >= N_MIN;
                        W.cstate[t] = acc ? CS_ACCEPTED : CS_REJECTED;
                        W.seg_n[t] = acc ? sure : 0;
                    } else if (sure + unk < N_MIN) {
                        W.cstate[t] = CS_REJECTED;
                        W.seg_n[t] = 0;
                    } else {
                        s_undecided = 1;
                    }
                }
            }
            __syncthreads();
            more = s_undecided != 0;
            __syncthreads();
        }
        round -= 1;
        if (threadIdx.x == 0) {
            if (more) set_status(W, ST_TIMEOUT);
            atomicMax(W.counters + CNT_ROUNDS, round);
        }
        // rejected up front, or left undecided by a timeout: no kept hits
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
            const int st = W.cstate[t];
            if (st == CS_UNDECIDED || (st == CS_REJECTED && W.cand_n[t] < N_MIN)) W.seg_n[t] = 0;
        }
        __syncthreads();
    }
}

}  // namespace

void launch_select(const Work &W, cudaStream_t s) {
    const int block = W.tune.block[4] > 0 ? W.tune.block[4] : 1024;
    int grid = W.tune.grid[4] > 0 ? W.tune.grid[4] : W.sm_count * 2;
    const int items = W.n_events * W.ns;
    if (grid > items) grid = items > 0 ? items : 1;
    k_select<<<grid, block, 0, s>>>(W);
}

}  // namespace tpc
