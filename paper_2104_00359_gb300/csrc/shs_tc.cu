// Diagnostic entry point for the tensor-core machinery used by the
// reduced-precision tails: one CTA computes D = A B^T (M = 128) with tcgen05
// MMAs accumulating in tensor memory: plain BF16 (mode 0), BF16 split in two
// parts (mode 1: A_hi B_hi + A_lo B_hi + A_hi B_lo), and the tails' operand
// types (modes 2-4: BF16 in three parts, TF32 in two, FP16 in two).

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

// Split-precision self-test (modes 2-4): A [128 x KD] and B [n x KD] split
// into the parts of the operand type, every product term of the precision.
template <int PR, int KD>
__global__ void __launch_bounds__(128) tc_split_selftest_kernel(const float* A, const float* B, int N, float* D,
                                                                int* status) {
    using P = shs::tc::Prec<PR>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t a_part = kM * KD * P::kElem, b_part = static_cast<uint32_t>(N) * KD * P::kElem;
    unsigned char* sA = smem;
    unsigned char* sB = smem + P::kParts * a_part;
    {
        float v[KD];
        for (int k = 0; k < KD; ++k) v[k] = A[tid * KD + k];
        shs::tc::store_row_split<PR, KD>(sA, a_part, tid, v);
    }
    for (int n = tid; n < N; n += 128) {
        float v[KD];
        for (int k = 0; k < KD; ++k) v[k] = B[n * KD + k];
        shs::tc::store_row_split<PR, KD>(sB, b_part, n, v);
    }
    if (warp == 0) shs::tc::tmem_alloc(&tmem_base, 256);
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
        // parts of B sit b_part = N KD eb bytes apart: the issue loop below
        // spells out the generic form (run-time part strides)
        constexpr uint32_t T = 16 / P::kElem;
        constexpr uint32_t SBO = (KD / T) * 128;
        const uint32_t idesc = shs::tc::idesc_of<PR>(kM, N);
        for (int t = 0; t < P::kTerms; ++t)
            for (int ks = 0; ks < KD / P::kKmma; ++ks) {
                const uint64_t ad = shs::tc::make_desc(shs::tc::smem_u32(sA) + shs::tc::term_a<PR>(t) * a_part + ks * 256, SBO);
                const uint64_t bd = shs::tc::make_desc(shs::tc::smem_u32(sB) + shs::tc::term_b<PR>(t) * b_part + ks * 256, SBO);
                shs::tc::mma<PR>(tmem, ad, bd, idesc, t > 0 || ks > 0);
            }
        shs::tc::commit(&bar);
    }
    const bool ok = shs::tc::mbar_wait(&bar, 0);
    if (!ok && tid == 0) atomicExch(status, shs::kDevTimeout);
    shs::tc::fence_after_sync();
    if (ok) {
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
        for (int c = 0; c < N; c += 16) {
            float v[16];
            shs::tc::tmem_ld16(lane_addr + c, v);
            for (int i = 0; i < 16; ++i) D[tid * N + c + i] = v[i];
        }
    }
    shs::tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) shs::tc::tmem_dealloc(tmem, 256);
}

// As above with A in tensor memory (modes 5-7): the split rows are stored by
// each thread into its lane from column 256, the MMAs read A from there.
template <int PR, int KD>
__global__ void __launch_bounds__(128) tc_split_ts_selftest_kernel(const float* A, const float* B, int N, float* D,
                                                                   int* status) {
    using P = shs::tc::Prec<PR>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t b_part = static_cast<uint32_t>(N) * KD * P::kElem;
    constexpr uint32_t a_cols = shs::tc::tmem_cols<PR>(KD);
    unsigned char* sB = smem;
    for (int n = tid; n < N; n += 128) {
        float v[KD];
        for (int k = 0; k < KD; ++k) v[k] = B[n * KD + k];
        shs::tc::store_row_split<PR, KD>(sB, b_part, n, v);
    }
    if (warp == 0) shs::tc::tmem_alloc(&tmem_base, 512);
    if (tid == 0) {
        shs::tc::mbar_init1(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    shs::tc::fence_before_sync();
    __syncthreads();
    shs::tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_addr = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    {
        float v[KD];
        for (int k = 0; k < KD; ++k) v[k] = A[tid * KD + k];
        shs::tc::tmem_store_split<PR, KD>(lane_addr + 256, a_cols, 0, v);
        shs::tc::tmem_wait_st();
    }
    shs::tc::fence_async_smem();
    shs::tc::fence_before_sync();
    __syncthreads();
    shs::tc::fence_after_sync();
    if (tid == 0) {
        constexpr uint32_t T = 16 / P::kElem;
        constexpr uint32_t SBO = (KD / T) * 128;
        const uint32_t idesc = shs::tc::idesc_of<PR>(kM, N);
        for (int t = 0; t < P::kTerms; ++t)
            for (int ks = 0; ks < KD / P::kKmma; ++ks) {
                const uint64_t bd = shs::tc::make_desc(shs::tc::smem_u32(sB) + shs::tc::term_b<PR>(t) * b_part + ks * 256, SBO);
                shs::tc::mma_ts<PR>(tmem, tmem + 256 + shs::tc::term_a<PR>(t) * a_cols + ks * 8, bd, idesc, t > 0 || ks > 0);
            }
        shs::tc::commit(&bar);
    }
    const bool ok = shs::tc::mbar_wait(&bar, 0);
    if (!ok && tid == 0) atomicExch(status, shs::kDevTimeout);
    shs::tc::fence_after_sync();
    if (ok) {
        for (int c = 0; c < N; c += 16) {
            float v[16];
            shs::tc::tmem_ld16(lane_addr + c, v);
            for (int i = 0; i < 16; ++i) D[tid * N + c + i] = v[i];
        }
    }
    shs::tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) shs::tc::tmem_dealloc(tmem, 512);
}

template <int PR, int KD>
cudaError_t launch_split_ts_selftest(const float* A, const float* B, int n, float* D, int* status, cudaStream_t s) {
    using P = shs::tc::Prec<PR>;
    const size_t smem = static_cast<size_t>(P::kParts) * P::kElem * KD * n;
    auto kern = tc_split_ts_selftest_kernel<PR, KD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<1, 128, smem, s>>>(A, B, n, D, status);
    shs::count_launch();
    return cudaGetLastError();
}

template <int PR, int KD>
cudaError_t launch_split_selftest(const float* A, const float* B, int n, float* D, int* status, cudaStream_t s) {
    using P = shs::tc::Prec<PR>;
    const size_t smem = static_cast<size_t>(P::kParts) * P::kElem * KD * (kM + n);
    auto kern = tc_split_selftest_kernel<PR, KD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<1, 128, smem, s>>>(A, B, n, D, status);
    shs::count_launch();
    return cudaGetLastError();
}

template <int PR>
cudaError_t split_selftest(const float* A, const float* B, int n, int k, bool ts, float* D, int* status,
                           cudaStream_t s) {
    switch (k) {
        case 16: return ts ? launch_split_ts_selftest<PR, 16>(A, B, n, D, status, s)
                           : launch_split_selftest<PR, 16>(A, B, n, D, status, s);
        case 32: return ts ? launch_split_ts_selftest<PR, 32>(A, B, n, D, status, s)
                           : launch_split_selftest<PR, 32>(A, B, n, D, status, s);
        case 64: return ts ? launch_split_ts_selftest<PR, 64>(A, B, n, D, status, s)
                           : launch_split_selftest<PR, 64>(A, B, n, D, status, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

extern "C" shs_status shs_tc_gemm_selftest(const float* A, const float* B, int32_t n, int32_t k, int32_t split,
                                           float* D, int32_t* device_status, void* stream) {
    if (!A || !B || !D || !device_status)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL argument"));
    if (n < 16 || n > kMaxN || n % 16 || k < 16 || k > kMaxKdim || k % 16)
        return static_cast<shs_status>(shs::report_error(
            SHS_ERR_INVALID_ARG, "tc self-test needs 16 <= n <= 256, 16 <= k <= 64, multiples of 16"));
    if (split < 0 || split > 7)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "tc self-test mode %d not in 0..7", split));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (split >= 2) {
        if (k == 48) return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "split modes take k = 16, 32 or 64"));
        const bool ts = split >= 5;
        const int m = ts ? split - 3 : split;
        if (m == 2) e = split_selftest<shs::tc::kPrecBF16>(A, B, n, k, ts, D, device_status, st);
        else if (m == 3) e = split_selftest<shs::tc::kPrecTF32>(A, B, n, k, ts, D, device_status, st);
        else e = split_selftest<shs::tc::kPrecFP16>(A, B, n, k, ts, D, device_status, st);
        return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, "tc self-test launch"));
    }
    const size_t smem = 2 * (static_cast<size_t>(kM) * k * 2) + 2 * (static_cast<size_t>(n) * k * 2);
    e = cudaFuncSetAttribute(tc_gemm_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
    if (e != cudaSuccess) return static_cast<shs_status>(shs::report_cuda(e, "tc self-test attribute"));
    tc_gemm_selftest_kernel<<<1, 128, smem, st>>>(A, B, n, k, split ? 1 : 0, D, device_status);
    shs::count_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, "tc self-test launch"));
}
