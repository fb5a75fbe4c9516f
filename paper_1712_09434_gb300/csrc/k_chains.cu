// S3 link cleaning and S4 chains (seeds of the cellular automaton; arxiv 1712.09434 section 3:
// short track candidates of "around 5 to 10 hits" built from neighbour links).
//
// A link c -> u is kept only if it is mutual (down[u] == c); both directions read the uncleaned
// arrays, so the cleaning is computed on the fly and never stored.  A chain starts at a cluster
// with a kept up-link and no kept down-link and follows the kept up-links; chains of at least
// N_SEED hits are compacted in start-cluster order: per-bin counts (one warp per bin), a
// device-wide scan, and an ordered warp-ballot compaction.
#include "tpc_common.cuh"

namespace tpc {

namespace {

__device__ __forceinline__ bool mutual_up(const Work &W, int c, int *u_out) {
    const int u = W.up[c];
    *u_out = u;
    return u >= 0 && W.down[u] == c;
}

// chain length from a start cluster, or 0 if c is not a start
__device__ int chain_length(const Work &W, int c, int max_len) {
    int u;
    if (!mutual_up(W, c, &u)) return 0;
    const int d = W.down[c];
    if (d >= 0 && W.up[d] == c) return 0;    // has a kept down-link: not a start
    int len = 1, x = c;
    while (len < max_len) {
        int nx;
        if (!mutual_up(W, x, &nx)) break;
        x = nx;
        len++;
    }
    return len;
}

__global__ void __launch_bounds__(256) k_chain_count(Work W) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int max_len = W.geom->n_rows;
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < W.nbins; b += nw) {
        const int c0 = W.bin_off[b], c1 = W.bin_off[b + 1];
        int cnt = 0;
        for (int c = c0 + lane; c < c1; c += 32) {
            int len = chain_length(W, c, max_len);
            if (len < N_SEED) len = 0;
            W.clen[c] = len;
            cnt += len > 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) W.bin_cnt[b] = cnt;
    }
}

__global__ void __launch_bounds__(256) k_chain_write(Work W) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < W.nbins; b += nw) {
        const int c0 = W.bin_off[b], c1 = W.bin_off[b + 1];
        int pos = W.chain_off[b];
        for (int base = c0; base < c1; base += 32) {
            const int c = base + lane;
            const int len = c < c1 ? W.clen[c] : 0;
            const unsigned m = __ballot_sync(0xffffffffu, len > 0);
            if (len > 0) {
                const int p = pos + __popc(m & ((1u << lane) - 1u));
                if (p < W.cap_chains) {
                    W.chain_start[p] = c;
                    W.chain_len[p] = len;
                    W.chain_bin[p] = b;
                } else {
                    set_status(W, ST_CAPACITY);
                }
            }
            pos += __popc(m);
        }
    }
}

}  // namespace

void launch_chains(const Work &W, cudaStream_t s) {
    const int block = W.tune.block[2] > 0 ? W.tune.block[2] : 256;
    const int warps = block / 32;
    int grid = (W.nbins + warps - 1) / warps;
    if (W.tune.grid[2] > 0 && grid > W.tune.grid[2]) grid = W.tune.grid[2];
    if (grid < 1) grid = 1;
    k_chain_count<<<grid, block, 0, s>>>(W);
    scan_exclusive(W.bin_cnt, W.chain_off, W.nbins, nullptr, W.counters + CNT_NCHAINS, W.scan_tmp,
                   W.scan_tmp_len, s);
    k_chain_write<<<grid, block, 0, s>>>(W);
}

}  // namespace tpc
