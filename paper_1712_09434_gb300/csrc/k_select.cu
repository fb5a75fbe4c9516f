// S6 track selection: the exact result of the sequential greedy rule, computed in parallel rounds.
//
// Sequential rule: candidates in priority order (more hits first, then earlier seed) keep the hits
// that no already-accepted candidate owns and are accepted with at least N_MIN kept hits.  Hits
// belong to one sector, so one CTA handles one (event, sector) from a work queue.  Priority key
// (unique, smaller = earlier): ((n_rows - n_hits) << 23) | (candidate index in the sector).
//
// Round: every undecided candidate claims its hits (atomicMax on (round << 32 | ~key), so the
// latest round wins and inside it the smallest key); an undecided candidate whose hits are all
// resolved (owned by an accepted candidate = lost, or claimed by itself = kept) decides; one that
// cannot reach N_MIN even with its unresolved hits is rejected.  Newly accepted candidates then
// take ownership of their kept hits.  The highest-priority undecided candidate always decides, so
// the rounds end, and every decision equals the sequential one (a candidate decides only when no
// higher-priority undecided candidate shares a hit with it).
#include "tpc_common.cuh"

namespace tpc {

namespace {

enum { CS_UNDECIDED = 0, CS_ACCEPT_NEW = 1, CS_ACCEPTED = 2, CS_REJECTED = 3 };

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
        int round = 1;
        for (; round <= SELECT_MAX_ROUNDS; round++) {
            // claims
            for (int t = t0 + warp; t < t1; t += nwarps) {
                if (W.cstate[t] != CS_UNDECIDED) continue;
                const unsigned long long v =
                    ((unsigned long long)round << 32) | (uint32_t)~key_of(nr, W.cand_n[t], t - t0);
                const int rr = W.cand_rows[t];
                const int32_t *sl = W.cand_slots + (size_t)t * nr;
                for (int r = (rr & 0xffff) + lane; r <= (rr >> 16); r += 32) {
                    const int h = sl[r];
                    if (h >= 0) atomicMax(claim + h, v);
                }
            }
            if (threadIdx.x == 0) s_undecided = 0;
            __syncthreads();
            // decisions
            for (int t = t0 + warp; t < t1; t += nwarps) {
                if (W.cstate[t] != CS_UNDECIDED) continue;
                const uint32_t key = key_of(nr, W.cand_n[t], t - t0);
                const int rr = W.cand_rows[t];
                const int32_t *sl = W.cand_slots + (size_t)t * nr;
                int sure = 0, unk = 0;
                for (int r = (rr & 0xffff) + lane; r <= (rr >> 16); r += 32) {
                    const int h = sl[r];
                    if (h < 0 || W.owner[h] != KEY_NONE) continue;       // miss, or lost
                    const unsigned long long v = claim[h];
                    if ((int)(v >> 32) == round && (uint32_t)~(uint32_t)v == key) sure++; else unk++;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sure += __shfl_xor_sync(0xffffffffu, sure, o);
                    unk += __shfl_xor_sync(0xffffffffu, unk, o);
                }
                if (lane == 0) {
                    if (unk == 0)
                        W.cstate[t] = sure >= N_MIN ? CS_ACCEPT_NEW : CS_REJECTED;
                    else if (sure + unk < N_MIN)
                        W.cstate[t] = CS_REJECTED;
                    else
                        s_undecided = 1;
                }
            }
            __syncthreads();
            // ownership of the newly accepted
            for (int t = t0 + warp; t < t1; t += nwarps) {
                if (W.cstate[t] != CS_ACCEPT_NEW) continue;
                const uint32_t key = key_of(nr, W.cand_n[t], t - t0);
                const unsigned long long v = ((unsigned long long)round << 32) | (uint32_t)~key;
                const int rr = W.cand_rows[t];
                const int32_t *sl = W.cand_slots + (size_t)t * nr;
                for (int r = (rr & 0xffff) + lane; r <= (rr >> 16); r += 32) {
                    const int h = sl[r];
                    if (h >= 0 && W.owner[h] == KEY_NONE && claim[h] == v) W.owner[h] = key;
                }
                __syncwarp();
                if (lane == 0) W.cstate[t] = CS_ACCEPTED;
            }
            const int undecided = s_undecided;
            __syncthreads();
            if (!undecided) break;
        }
        if (threadIdx.x == 0) {
            if (round > SELECT_MAX_ROUNDS) set_status(W, ST_TIMEOUT);
            atomicMax(W.counters + CNT_ROUNDS, round);
        }
        // kept hits per candidate
        for (int t = t0 + warp; t < t1; t += nwarps) {
            int kept = 0;
            if (W.cstate[t] == CS_ACCEPTED) {
                const uint32_t key = key_of(nr, W.cand_n[t], t - t0);
                const int rr = W.cand_rows[t];
                const int32_t *sl = W.cand_slots + (size_t)t * nr;
                for (int r = (rr & 0xffff) + lane; r <= (rr >> 16); r += 32) {
                    const int h = sl[r];
                    kept += h >= 0 && W.owner[h] == key;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
            }
            if (lane == 0) W.seg_n[t] = kept;
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
