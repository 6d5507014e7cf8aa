// Diagnostic: the FP32 fused multiply-add throughput the shading kernels are
// measured against.  Every thread runs kChains independent FMA chains of
// `iters` steps; the chains' sum is stored so that nothing is eliminated.

#include <cstdint>
#include <cuda_runtime.h>

#include "shs.h"
#include "shs_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fma_peak_kernel(int64_t iters, float* out) {
    float x[kChains];
    const float a = 1.0f - 1e-7f * (threadIdx.x & 7), b = 1e-7f * (blockIdx.x & 15);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = static_cast<float>(threadIdx.x + c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" shs_status shs_fp32_fma_probe(int32_t blocks, int64_t iters, float* out, void* stream) {
    if (blocks < 1 || blocks > (1 << 20) || iters < 1 || !out)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "blocks in 1..2^20, iters >= 1, out"));
    fma_peak_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(iters, out);
    shs::count_launch();
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, "fma probe"));
}
