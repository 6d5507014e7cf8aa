// Diagnostic entry point for the tensor-core machinery used by the
// reduced-precision tail: one CTA computes D = A B^T (M = 128) with tcgen05
// BF16 MMAs accumulating in tensor memory, optionally in split precision
// (A ~ A_hi + A_lo, B ~ B_hi + B_lo, D = A_hi B_hi + A_lo B_hi + A_hi B_lo).

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "shs.h"
#include "shs_internal.h"
#include "shs_tc.cuh"

namespace {

constexpr int kM = 128;
constexpr int kMaxKdim = 64;
constexpr int kMaxN = 256;

__global__ void __launch_bounds__(128) tc_gemm_selftest_kernel(const float* A, const float* B, int N, int Kdim,
                                                               int split, float* D, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t a_bytes = kM * Kdim * 2, b_bytes = N * Kdim * 2;
    unsigned char* sAh = smem;
    unsigned char* sAl = sAh + a_bytes;
    unsigned char* sBh = sAl + a_bytes;
    unsigned char* sBl = sBh + b_bytes;
    for (int k = 0; k < Kdim; ++k) {
        uint16_t h, l;
        shs::tc::split_bf16(A[tid * Kdim + k], h, l);
        const uint32_t o = shs::tc::kmajor_offset(tid, k, Kdim);
        *reinterpret_cast<uint16_t*>(sAh + o) = h;
        *reinterpret_cast<uint16_t*>(sAl + o) = l;
    }
    for (int e = tid; e < N * Kdim; e += 128) {
        const int n = e / Kdim, k = e % Kdim;
        uint16_t h, l;
        shs::tc::split_bf16(B[e], h, l);
        const uint32_t o = shs::tc::kmajor_offset(n, k, Kdim);
        *reinterpret_cast<uint16_t*>(sBh + o) = h;
        *reinterpret_cast<uint16_t*>(sBl + o) = l;
    }
    uint32_t ncols = 32;
    while (ncols < static_cast<uint32_t>(N)) ncols <<= 1;
    if (warp == 0) shs::tc::tmem_alloc(&tmem_base, ncols);
    if (tid == 0) {
        shs::tc::mbar_init1(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    shs::tc::fence_async_smem();
    shs::tc::fence_before_sync();
    __syncthreads();
    shs::tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        const uint32_t idesc = shs::tc::idesc_bf16(kM, N);
        const uint32_t sbo = (Kdim / 8) * 128;
        for (int ks = 0; ks < Kdim / 16; ++ks) {
            const uint32_t off = ks * 256;
            const uint64_t ah = shs::tc::make_desc(shs::tc::smem_u32(sAh) + off, sbo);
            const uint64_t al = shs::tc::make_desc(shs::tc::smem_u32(sAl) + off, sbo);
            const uint64_t bh = shs::tc::make_desc(shs::tc::smem_u32(sBh) + off, sbo);
            const uint64_t bl = shs::tc::make_desc(shs::tc::smem_u32(sBl) + off, sbo);
            shs::tc::mma_bf16(tmem, ah, bh, idesc, ks > 0);
            if (split) {
                shs::tc::mma_bf16(tmem, al, bh, idesc, true);
                shs::tc::mma_bf16(tmem, ah, bl, idesc, true);
            }
        }
        shs::tc::commit(&bar);
    }
    const bool ok = shs::tc::mbar_wait(&bar, 0);
    if (!ok && tid == 0) atomicExch(status, shs::kDevTimeout);
    shs::tc::fence_after_sync();
    if (ok) {
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
        for (int c = 0; c < N; c += 32) {
            float v[32];
            shs::tc::tmem_ld32(lane_addr + c, v);
            for (int i = 0; i < 32 && c + i < N; ++i) D[tid * N + c + i] = v[i];
        }
    }
    shs::tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) shs::tc::tmem_dealloc(tmem, ncols);
}

__global__ void pack_split_kernel(const float* src, int rows, int cols, int fp16, uint16_t* hi, uint16_t* lo) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    const int r = e / cols, c = e % cols;
    uint16_t h, l;
    if (fp16) shs::tc::split_fp16(src[e], h, l);
    else shs::tc::split_bf16(src[e], h, l);
    const uint32_t o = shs::tc::kmajor_offset(r, c, cols) >> 1;
    hi[o] = h;
    lo[o] = l;
}

}  // namespace

namespace shs {
cudaError_t launch_pack_split(const float* src, int rows, int cols, int fp16, void* hi, void* lo, cudaStream_t s) {
    const int n = rows * cols;
    pack_split_kernel<<<(n + 255) / 256, 256, 0, s>>>(src, rows, cols, fp16, static_cast<uint16_t*>(hi),
                                                      static_cast<uint16_t*>(lo));
    count_launch();
    return cudaGetLastError();
}
}  // namespace shs

extern "C" shs_status shs_tc_gemm_selftest(const float* A, const float* B, int32_t n, int32_t k, int32_t split,
                                           float* D, int32_t* device_status, void* stream) {
    if (!A || !B || !D || !device_status)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL argument"));
    if (n < 16 || n > kMaxN || n % 16 || k < 16 || k > kMaxKdim || k % 16)
        return static_cast<shs_status>(shs::report_error(
            SHS_ERR_INVALID_ARG, "tc self-test needs 16 <= n <= 256, 16 <= k <= 64, multiples of 16"));
    const size_t smem = 2 * (static_cast<size_t>(kM) * k * 2) + 2 * (static_cast<size_t>(n) * k * 2);
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return static_cast<shs_status>(shs::report_cuda(e, "tc self-test attribute"));
    tc_gemm_selftest_kernel<<<1, 128, smem, static_cast<cudaStream_t>(stream)>>>(A, B, n, k, split ? 1 : 0, D,
                                                                              device_status);
    shs::count_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, "tc self-test launch"));
}
