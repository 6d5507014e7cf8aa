// Warp-level sums shared by the adjoint kernels.
#pragma once

#include <cuda_runtime.h>

namespace shs {
namespace {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV values (NV a power of two <= 32) over the warp by halving exchanges:
// afterwards v[0] on lane l holds the warp total of value (l >> (5 - log2 NV)).
template <int NV>
__device__ __forceinline__ void warp_transpose_sum(float* v, int lane) {
#pragma unroll
    for (int o = 16, cnt = NV; o > 0; o >>= 1) {
        if (cnt > 1) {
            const int half = cnt / 2;
            const bool up = lane & o;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const float send = up ? v[i] : v[i + half];
                const float keep = up ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
            cnt = half;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
}

constexpr int log2c(int v) { return v <= 1 ? 0 : 1 + log2c(v / 2); }
constexpr int pow2_at_least(int v) { return v <= 1 ? 1 : 2 * pow2_at_least((v + 1) / 2); }

// Add the warp totals of vals[0..NV) into dst[0..NV) (one lane per value).
template <int NV>
__device__ __forceinline__ void warp_sum_into(const float* vals, float* dst, int lane) {
#pragma unroll
    for (int base = 0; base < NV; base += 32) {
        const int rem = NV - base;
        if (rem >= 32) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = vals[base + i];
            warp_transpose_sum<32>(v, lane);
            dst[base + lane] += v[0];
        } else {
            constexpr int R = NV % 32 == 0 ? 32 : NV % 32;
            constexpr int RP = pow2_at_least(R);
            float v[RP];
#pragma unroll
            for (int i = 0; i < RP; ++i) v[i] = i < R ? vals[base + i] : 0.f;
            warp_transpose_sum<RP>(v, lane);
            constexpr int sh = 5 - log2c(RP);
            const int idx = lane >> sh;
            if ((lane & ((1 << sh) - 1)) == 0 && idx < R) dst[base + idx] += v[0];
        }
    }
}

}  // namespace
}  // namespace shs
