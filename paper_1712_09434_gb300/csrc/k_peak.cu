// FP32 fused multiply-add throughput of the GPU: the roof that the Kalman refit and its adjoint
// (FP32 arithmetic per thread, no tensor cores) are measured against.  The paper has no
// counterpart; this is a diagnostic of the library.
//
// Every thread runs 8 independent chains x <- x * a + b in registers (enough independent work per
// warp to keep the FMA pipes busy at a few warps per scheduler); the constants keep the values
// finite and the final sum is stored so that no chain can be removed.
#include "tpc_common.cuh"

namespace tpc {
namespace {

constexpr int FMA_CHAINS = 8;
constexpr int FMA_UNROLL = 16;

__global__ void __launch_bounds__(256) k_fma_peak(float *out, long long iters, float a, float b) {
    float x[FMA_CHAINS];
#pragma unroll
    for (int j = 0; j < FMA_CHAINS; j++) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (long long i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < FMA_UNROLL; u++) {
#pragma unroll
            for (int j = 0; j < FMA_CHAINS; j++) x[j] = fmaf(x[j], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < FMA_CHAINS; j++) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace tpc

extern "C" int tpc_fma_peak(float *out, int64_t iters, int32_t ctas_per_sm, int32_t threads, int64_t *flops,
                            void *stream) {
    if (!out || !flops || iters < 1 || ctas_per_sm < 1 || ctas_per_sm > 64 || threads < 32 || threads > 256 ||
        threads % 32)
        return TPC_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return TPC_ERR_CUDA;
    const long long grid = (long long)sms * ctas_per_sm;
    *flops = 2ll * grid * threads * iters * tpc::FMA_UNROLL * tpc::FMA_CHAINS;
    tpc::k_fma_peak<<<(unsigned)grid, threads, 0, static_cast<cudaStream_t>(stream)>>>(out, iters, 0.999999f, 1e-7f);
    return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}
