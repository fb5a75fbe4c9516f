// Device-wide exclusive scan of int32 counts (reduce / scan tile sums / apply).  Used to turn
// per-bin chain counts into chain offsets, head flags into track ids and per-track hit counts
// into hit offsets, all without a host round trip (counts stay on the device).
#include "tpc_common.cuh"

namespace tpc {

namespace {

constexpr int SB = 256;           // threads per scan block
constexpr int SI = 8;             // items per thread
constexpr int TILE = SB * SI;

__device__ __forceinline__ int warp_incl(int v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one value per thread across the block; the block total goes to *tot
__device__ int block_excl(int v, int *tot) {
    __shared__ int ws[SB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int inc = warp_incl(v);
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int x = lane < SB / 32 ? ws[lane] : 0;
        const int xi = warp_incl(x);
        if (lane < SB / 32) ws[lane] = xi - x;
        if (lane == 31) *tot = xi;
    }
    __syncthreads();
    const int r = ws[w] + inc - v;
    __syncthreads();
    return r;
}

__device__ __forceinline__ int resolve_n(int n_cap, const int32_t *n_dev) {
    if (!n_dev) return n_cap;
    int n = *n_dev;
    return n < 0 ? 0 : (n > n_cap ? n_cap : n);
}

__global__ void k_scan_reduce(const int32_t *__restrict__ in, int n_cap, const int32_t *n_dev,
                              int32_t *__restrict__ tile_sum) {
    int n = resolve_n(n_cap, n_dev);
    long long base = (long long)blockIdx.x * TILE;
    int s = 0;
    if (base < n) {
        for (int k = 0; k < SI; k++) {
            long long i = base + (long long)k * SB + threadIdx.x;
            if (i < n) s += in[i];
        }
    }
    __shared__ int tot;
    block_excl(s, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = base < n ? tot : 0;
}

__global__ void k_scan_tiles(int32_t *__restrict__ tile_sum, int n_tiles, int n_cap, const int32_t *n_dev,
                             int32_t *__restrict__ out, int32_t *total_dev) {
    __shared__ int tot;
    int carry = 0;
    for (int b0 = 0; b0 < n_tiles; b0 += SB) {
        int i = b0 + threadIdx.x;
        int v = i < n_tiles ? tile_sum[i] : 0;
        int e = block_excl(v, &tot);
        if (i < n_tiles) tile_sum[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int n = resolve_n(n_cap, n_dev);
        out[n] = carry;
        if (total_dev) *total_dev = carry;
    }
}

__global__ void k_scan_apply(const int32_t *__restrict__ in, int32_t *__restrict__ out, int n_cap,
                             const int32_t *n_dev, const int32_t *__restrict__ tile_off) {
    int n = resolve_n(n_cap, n_dev);
    long long base = (long long)blockIdx.x * TILE;
    if (base >= n) return;
    __shared__ int tot;
    // each thread owns SI consecutive items
    long long i0 = base + (long long)threadIdx.x * SI;
    int v[SI];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SI; k++) {
        long long i = i0 + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int e = block_excl(s, &tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SI; k++) {
        long long i = i0 + k;
        if (i < n) out[i] = e;
        e += v[k];
    }
}

}  // namespace

int scan_tmp_needed(int n_cap) { return (n_cap + TILE - 1) / TILE + 1; }

void scan_exclusive(const int32_t *in, int32_t *out, int n_cap, const int32_t *n_dev, int32_t *total_dev,
                    int32_t *tmp, int tmp_len, cudaStream_t s) {
    int n_tiles = (n_cap + TILE - 1) / TILE;
    if (n_tiles < 1) n_tiles = 1;
    (void)tmp_len;
    k_scan_reduce<<<n_tiles, SB, 0, s>>>(in, n_cap, n_dev, tmp);
    k_scan_tiles<<<1, SB, 0, s>>>(tmp, n_tiles, n_cap, n_dev, out, total_dev);
    k_scan_apply<<<n_tiles, SB, 0, s>>>(in, out, n_cap, n_dev, tmp);
}

}  // namespace tpc
