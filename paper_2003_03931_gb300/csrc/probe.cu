// probe.cu -- FP32 fused multiply-add throughput of the GPU at hand: the
// peak against which the tile pass (bound by FP32 issue, not by memory) is
// measured.  Each thread runs kChains independent FMA chains so that every
// sub-partition has enough independent instructions to issue one FMA per
// cycle; the chains are summed into one output word per thread so nothing
// is dead code.
#include "pmpm_impl.cuh"

namespace pmpm {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(float* __restrict__ out, int iters,
                                                             float b, float c) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace pmpm

extern "C" int pmpm_probe_fma(float* d_out, int64_t out_len, void* stream, int32_t iters,
                              double* flops, float* ms) {
    using namespace pmpm;
    if (!d_out || !flops || !ms || iters < 1 || out_len < kProbeThreads || out_len % kProbeThreads ||
        out_len / kProbeThreads > 0x7fffffff)
        return PMPM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PMPM_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PMPM_ECUDA;
    }
    const int blocks = (int)(out_len / kProbeThreads);
    cudaEventRecord(e0, st);
    k_fma_probe<<<blocks, kProbeThreads, 0, st>>>(d_out, iters, 0.99999994f, 1e-7f);
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return PMPM_ECUDA;
    *ms = t;
    *flops = 2.0 * kChains * (double)iters * (double)out_len;
    return PMPM_OK;
}
