// S3 link cleaning and S4 chains (seeds of the cellular automaton; arxiv 1712.09434 section 3:
// short track candidates of five to ten hits built from neighbour links).
//
// A link c -> u is kept only if it is mutual (down[u] == c); both directions read the uncleaned
// arrays.  The kept up-links are written once, with their 2- and 4-link successors (pointer
// jumping), so that a chain walk takes four links per dependent load.  A chain starts at a cluster
// with a kept up-link and no kept down-link and follows the kept up-links; chains of at least
// N_SEED hits are compacted in start-cluster order: per-bin counts (one warp per bin), a
// device-wide scan, and an ordered warp-ballot compaction.
#include "tpc_common.cuh"

namespace tpc {

namespace {

// Kept up-link of every cluster (-1 if none or not mutual), and the successors 2 and 4 links
// further: a chain walk then takes four links per dependent load.  The arrays live in the
// selection's claim and owner words, which the selection re-initialises before use.
struct Jumps {
    int32_t *n1, *n2, *n4;
};
__device__ __forceinline__ Jumps jumps_of(const Work &W) {
    Jumps j;
    j.n1 = reinterpret_cast<int32_t *>(W.claim);
    j.n2 = reinterpret_cast<int32_t *>(W.claim) + (W.n_clusters + 1);
    j.n4 = reinterpret_cast<int32_t *>(W.owner);
    return j;
}

__global__ void k_mutual(Work W) {
    const Jumps J = jumps_of(W);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < W.n_clusters; c += gridDim.x * blockDim.x) {
        const int u = W.up[c];
        J.n1[c] = u >= 0 && W.down[u] == c ? u : -1;
    }
}

__global__ void k_jump(Work W, const int32_t *src, int32_t *dst) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < W.n_clusters; c += gridDim.x * blockDim.x) {
        const int u = src[c];
        dst[c] = u >= 0 ? src[u] : -1;
    }
}

// chain length from a start cluster, or 0 if c is not a start (a start has a kept up-link and no
// kept down-link); the count of clusters along the kept up-links, at most max_len
__device__ int chain_length(const Work &W, const Jumps &J, int c, int max_len) {
    if (J.n1[c] < 0) return 0;
    const int d = W.down[c];
    if (d >= 0 && J.n1[d] == c) return 0;
    int len = 1, x = c;
    while (len < max_len) {
        if (len + 4 <= max_len) {
            const int y = J.n4[x];
            if (y >= 0) { x = y; len += 4; continue; }
        }
        if (len + 2 <= max_len) {
            const int y = J.n2[x];
            if (y >= 0) { x = y; len += 2; continue; }
        }
        const int y = J.n1[x];
        if (y < 0) break;
        x = y;
        len++;
    }
    return len;
}

__global__ void __launch_bounds__(256) k_chain_count(Work W) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int max_len = W.geom->n_rows;
    const Jumps J = jumps_of(W);
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < W.nbins; b += nw) {
        const int c0 = W.bin_off[b], c1 = W.bin_off[b + 1];
        int cnt = 0;
        for (int c = c0 + lane; c < c1; c += 32) {
            int len = chain_length(W, J, c, max_len);
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
    const int gj = W.sm_count * 8;
    k_mutual<<<gj, 256, 0, s>>>(W);
    int32_t *n1 = reinterpret_cast<int32_t *>(W.claim), *n2 = n1 + (W.n_clusters + 1);
    k_jump<<<gj, 256, 0, s>>>(W, n1, n2);
    k_jump<<<gj, 256, 0, s>>>(W, n2, reinterpret_cast<int32_t *>(W.owner));
    k_chain_count<<<grid, block, 0, s>>>(W);
    scan_exclusive(W.bin_cnt, W.chain_off, W.nbins, nullptr, W.counters + CNT_NCHAINS, W.scan_tmp,
                   W.scan_tmp_len, s);
    k_chain_write<<<grid, block, 0, s>>>(W);
}

}  // namespace tpc
