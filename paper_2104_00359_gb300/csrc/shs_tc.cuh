// Fifth-generation tensor-core helpers (tcgen05, sm_100-family) written as
// inline PTX: tensor-memory allocation, shared-memory matrix descriptors for
// the no-swizzle K-major canonical layout, the single-CTA BF16 MMA with FP32
// accumulation in tensor memory, completion through an mbarrier, and
// tensor-memory loads.
//
// Canonical K-major layout without swizzle (16-bit elements): the matrix is a
// grid of 8-row x 16-byte core matrices, each stored as 128 contiguous bytes.
// Element (r, k) of an R x Kdim operand lives at
//   (r / 8) * SBO + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// with SBO = (Kdim / 8) * 128: core matrices adjacent along K are 128 bytes
// apart (the descriptor's leading-dimension offset), 8-row groups are SBO
// apart (its stride-dimension offset).  One MMA consumes K = 16 (two core
// matrices along K); successive K steps advance the start address by 256 B.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace shs {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) in the canonical layout with Kdim columns.
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int kdim) {
    return static_cast<uint32_t>((r >> 3) * (kdim >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, LBO = 128 B, SBO, version 1,
// no swizzle.  Addresses and offsets are encoded in 16-byte units.
__device__ __forceinline__ uint64_t make_desc(uint32_t smem_addr, uint32_t sbo_bytes) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((smem_addr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>((128u >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo_bytes >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1u) << 46;          // descriptor version for tcgen05
    return d;                                      // base offset 0, no swizzle
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16 (fmt 1) or F16
// (fmt 0), both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16kind(int M, int N, uint32_t fmt) {
    return (1u << 4)                                // D format F32
         | (fmt << 7)                               // A format
         | (fmt << 10)                              // B format
         | (static_cast<uint32_t>(N >> 3) << 17)
         | (static_cast<uint32_t>(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) { return idesc_f16kind(M, N, 1u); }
__host__ __device__ constexpr uint32_t idesc_fp16(int M, int N) { return idesc_f16kind(M, N, 0u); }

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}

// Arrive on the mbarrier when every MMA this thread issued so far completes.
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Make this thread's generic-proxy shared-memory writes visible to the async proxy.
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Warp-wide: allocate ncols tensor-memory columns; the address goes to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(dst)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this thread's lane (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the mbarrier with a bound of about one second.
// Returns false when the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = now_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (ok) return true;
        if (now_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

// Bulk copy of `bytes` (multiple of 16) from global to shared memory that
// completes on `bar` (the caller arms the barrier with the expected bytes).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Round x to bfloat16 (nearest even) and return the remainder's bfloat16:
// x ~ hi + lo with about 16 significant bits.
__device__ __forceinline__ void split_bf16(float x, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

// Same split with IEEE half precision (11 significant bits per part).
__device__ __forceinline__ void split_fp16(float x, uint16_t& hi, uint16_t& lo) {
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(x - __half2float(h));
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(l);
}

template <bool FP16>
__device__ __forceinline__ void split16(float x, uint16_t& hi, uint16_t& lo) {
    if constexpr (FP16) split_fp16(x, hi, lo);
    else split_bf16(x, hi, lo);
}

// Store 64 values of row r as split 16-bit operands in the canonical K-major
// layout of a [rows x 64] operand (SBO = 1024 B).
template <bool FP16>
__device__ __forceinline__ void store_row64(unsigned char* hi_base, unsigned char* lo_base, int r, const float* v) {
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            uint16_t h0, l0, h1, l1;
            split16<FP16>(v[8 * g + 2 * e], h0, l0);
            split16<FP16>(v[8 * g + 2 * e + 1], h1, l1);
            h[e] = static_cast<uint32_t>(h0) | (static_cast<uint32_t>(h1) << 16);
            l[e] = static_cast<uint32_t>(l0) | (static_cast<uint32_t>(l1) << 16);
        }
        const uint32_t off = (r >> 3) * 1024 + g * 128 + (r & 7) * 16;
        *reinterpret_cast<uint4*>(hi_base + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo_base + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// ---------------------------------------------------------------------------
// Split-precision operands for the 8-band tensor-core tails.
//
// A float32 value x is carried as the sum of P parts of the MMA's input type:
// x ~ p_0 + p_1 + ..., p_j = rnd(x - p_0 - ... - p_{j-1}).  A product of
// split operands a b is the sum of the part products a_i b_j of total order
// i + j below the parts' count, each one MMA accumulating in float32 tensor
// memory, smallest first.
//   BF16: 3 parts per operand (about 24 significant bits), 6 products;
//   FP16: 2 parts (about 22 bits; operands pre-scaled into half range), 3;
//   TF32: 2 parts (about 22 bits), 3 products, K = 8 per MMA.
// An element pair (16-bit types) or element (TF32) fills 32 bits; 16 bytes of
// a row form one core-matrix row (8 elements of 16 bits, 4 of TF32), so the
// canonical K-major layout above holds for every type with the K index
// counted in 16-byte groups: element (r, k) of an R x KD operand with element
// size eb sits at (r / 8) SBO + (k / T) 128 + (r % 8) 16 + (k % T) eb,
// T = 16 / eb, SBO = (KD / T) 128.  One MMA consumes 32 bytes of K (K = 16
// for 16-bit types, 8 for TF32): successive K steps advance 256 bytes.
enum : int { kPrecBF16 = 0, kPrecFP16 = 1, kPrecTF32 = 2 };

template <int PR>
struct Prec;
template <>
struct Prec<kPrecBF16> {
    static constexpr int kElem = 2, kParts = 3, kKmma = 16, kTerms = 6;
    static constexpr uint32_t kFmt = 1;
};
template <>
struct Prec<kPrecFP16> {
    static constexpr int kElem = 2, kParts = 2, kKmma = 16, kTerms = 3;
    static constexpr uint32_t kFmt = 0;
};
template <>
struct Prec<kPrecTF32> {
    static constexpr int kElem = 4, kParts = 2, kKmma = 8, kTerms = 3;
    static constexpr uint32_t kFmt = 2;
};

// (part of A, part of B) of product term t, smallest first.
template <int PR>
__host__ __device__ constexpr int term_a(int t) {
    return Prec<PR>::kTerms == 6 ? (t == 0 ? 2 : t == 1 ? 1 : t == 2 ? 0 : t == 3 ? 1 : 0)
                                 : (t == 0 ? 1 : 0);
}
template <int PR>
__host__ __device__ constexpr int term_b(int t) {
    return Prec<PR>::kTerms == 6 ? (t == 0 ? 0 : t == 1 ? 1 : t == 2 ? 2 : t == 3 ? 0 : t == 4 ? 1 : 0)
                                 : (t == 1 ? 1 : 0);
}

// Instruction descriptor: D = F32, A = B of the precision's format, both
// K-major, M x N.
template <int PR>
__host__ __device__ constexpr uint32_t idesc_of(int M, int N) {
    return (1u << 4) | (Prec<PR>::kFmt << 7) | (Prec<PR>::kFmt << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

template <int PR>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                    bool accumulate) {
    if constexpr (PR == kPrecTF32) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
            ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u)
            : "memory");
    }
}

// D (+)= A B^T for split operands: A [128 x KD] and B [N x KD], both K-major
// with their parts `a_part` / `b_part` bytes apart; every product term of the
// precision over all K steps.  Issued by one thread.
// The descriptors of one GEMM differ only in their start address (the low
// 14-bit field, in 16-byte units): each is the first one plus a compile-time
// offset.  Shared-memory addresses stay below 256 KB, so the sum never
// carries out of the field.
template <int PR, int KD, uint32_t A_PART, uint32_t B_PART>
__device__ __forceinline__ void gemm_split(uint32_t d_tmem, uint32_t a_addr, uint32_t b_addr, uint32_t idesc,
                                           bool accumulate) {
    constexpr uint32_t T = 16 / Prec<PR>::kElem;
    constexpr uint32_t SBO = (KD / T) * 128;
    constexpr int KS = KD / Prec<PR>::kKmma;
    const uint64_t a0 = make_desc(a_addr, SBO), b0 = make_desc(b_addr, SBO);
#pragma unroll
    for (int t = 0; t < Prec<PR>::kTerms; ++t) {
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const uint64_t ad = a0 + ((term_a<PR>(t) * A_PART + ks * 256u) >> 4);
            const uint64_t bd = b0 + ((term_b<PR>(t) * B_PART + ks * 256u) >> 4);
            mma<PR>(d_tmem, ad, bd, idesc, accumulate || t > 0 || ks > 0);
        }
    }
}

// D (+)= A B^T with A [128 x K] in tensor memory (lane = row; 16-bit types
// two elements per 32-bit column, TF32 one), B from shared memory.
template <int PR>
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                       bool accumulate) {
    if constexpr (PR == kPrecTF32) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
            ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
            ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1u : 0u)
            : "memory");
    }
}

// Tensor-memory columns one part of a [128 x KD] operand takes.
template <int PR>
__host__ __device__ constexpr uint32_t tmem_cols(int KD) {
    return static_cast<uint32_t>(KD * Prec<PR>::kElem / 4);
}

// As gemm_split with the split A in tensor memory: part j of A starts at
// column a_tmem + j * A_COLS; one K step (32 bytes of K) takes 8 columns.
template <int PR, int KD, uint32_t A_COLS, uint32_t B_PART>
__device__ __forceinline__ void gemm_split_ts(uint32_t d_tmem, uint32_t a_tmem, uint32_t b_addr, uint32_t idesc,
                                              bool accumulate) {
    constexpr uint32_t T = 16 / Prec<PR>::kElem;
    constexpr uint32_t SBO = (KD / T) * 128;
    constexpr int KS = KD / Prec<PR>::kKmma;
    const uint64_t b0 = make_desc(b_addr, SBO);
#pragma unroll
    for (int t = 0; t < Prec<PR>::kTerms; ++t) {
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const uint64_t bd = b0 + ((term_b<PR>(t) * B_PART + ks * 256u) >> 4);
            mma_ts<PR>(d_tmem, a_tmem + term_a<PR>(t) * A_COLS + ks * 8u, bd, idesc, accumulate || t > 0 || ks > 0);
        }
    }
}

// Store 8 / 16 consecutive 32-bit columns of this thread's lane.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
                   "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Parts of x as raw bits (16-bit types in the low half).  BF16 and TF32
// parts are taken by truncation: p_0 keeps the leading 8 (BF16) or 11 (TF32)
// significant bits of x, and x - p_0 is exact in float32, so three BF16 parts
// hold x exactly; FP16 parts are rounded (a format conversion is needed).
template <int PR>
__device__ __forceinline__ void split_parts(float x, uint32_t* part) {
    float r = x;
#pragma unroll
    for (int j = 0; j < Prec<PR>::kParts; ++j) {
        if constexpr (PR == kPrecBF16) {
            const uint32_t u = __float_as_uint(r);
            part[j] = u >> 16;
            r -= __uint_as_float(u & 0xFFFF0000u);
        } else if constexpr (PR == kPrecFP16) {
            const __half h = __float2half_rn(r);
            part[j] = __half_as_ushort(h);
            r -= __half2float(h);
        } else {
            const uint32_t u = __float_as_uint(r) & 0xFFFFE000u;
            part[j] = u;
            r -= __uint_as_float(u);
        }
    }
}

// Store columns c0 .. c0 + NC - 1 (values v[0 .. NC)) of row r of a
// [rows x KD] split operand whose parts are `part_bytes` apart; c0 and NC are
// multiples of 16 bytes' worth of elements.
template <int PR, int KD, int NC>
__device__ __forceinline__ void store_cols_split(unsigned char* base, uint32_t part_bytes, int r, int c0,
                                                 const float* v) {
    constexpr int EB = Prec<PR>::kElem, T = 16 / EB, NP = Prec<PR>::kParts;
    constexpr uint32_t SBO = (KD / T) * 128;
    const uint32_t row_off = (r >> 3) * SBO + (r & 7) * 16 + (c0 / T) * 128;
#pragma unroll
    for (int g = 0; g < NC / T; ++g) {
        uint32_t w[NP][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if constexpr (EB == 2) {
                uint32_t lo[NP], hi[NP];
                split_parts<PR>(v[g * 8 + 2 * e], lo);
                split_parts<PR>(v[g * 8 + 2 * e + 1], hi);
#pragma unroll
                for (int j = 0; j < NP; ++j) w[j][e] = lo[j] | (hi[j] << 16);
            } else {
                uint32_t pp[NP];
                split_parts<PR>(v[g * 4 + e], pp);
#pragma unroll
                for (int j = 0; j < NP; ++j) w[j][e] = pp[j];
            }
        }
#pragma unroll
        for (int j = 0; j < NP; ++j)
            *reinterpret_cast<uint4*>(base + j * part_bytes + row_off + g * 128) =
                make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
    }
}

// Write NC values (this thread's row, from column c0 of the operand) of a
// split operand held in tensor memory: part j at column base + j * part_cols;
// NC * eb / 4 is a multiple of 8 columns.  Warp-collective; the caller waits
// (tmem_wait_st) before handing the operand to the MMA issuer.
template <int PR, int NC>
__device__ __forceinline__ void tmem_store_split(uint32_t lane_base, uint32_t part_cols, int c0, const float* v) {
    constexpr int EB = Prec<PR>::kElem, NP = Prec<PR>::kParts;
    constexpr int NW = NC * EB / 4;                 // 32-bit words per part
    static_assert(NW % 8 == 0, "whole 8-column stores");
    uint32_t w[NP][NW];
#pragma unroll
    for (int e = 0; e < NW; ++e) {
        if constexpr (EB == 2) {
            uint32_t lo[NP], hi[NP];
            split_parts<PR>(v[2 * e], lo);
            split_parts<PR>(v[2 * e + 1], hi);
#pragma unroll
            for (int j = 0; j < NP; ++j) w[j][e] = lo[j] | (hi[j] << 16);
        } else {
            uint32_t pp[NP];
            split_parts<PR>(v[e], pp);
#pragma unroll
            for (int j = 0; j < NP; ++j) w[j][e] = pp[j];
        }
    }
    const uint32_t col0 = static_cast<uint32_t>(c0 * EB / 4);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
#pragma unroll
        for (int q = 0; q < NW; q += 16) {
            if (NW - q >= 16) tmem_st16(lane_base + j * part_cols + col0 + q, &w[j][q]);
            else tmem_st8(lane_base + j * part_cols + col0 + q, &w[j][q]);
        }
    }
}

// Store row r (KD values) of a [rows x KD] split operand.
template <int PR, int KD>
__device__ __forceinline__ void store_row_split(unsigned char* base, uint32_t part_bytes, int r, const float* v) {
    store_cols_split<PR, KD, KD>(base, part_bytes, r, 0, v);
}

// 16 consecutive FP32 columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive FP32 columns of this thread's lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v) {
    static_assert(N % 8 == 0, "multiple of 8 columns");
    if constexpr (N % 32 == 0) {
#pragma unroll
        for (int c = 0; c < N; c += 32) tmem_ld32(taddr + c, v + c);
    } else if constexpr (N % 16 == 0) {
#pragma unroll
        for (int c = 0; c < N; c += 16) tmem_ld16(taddr + c, v + c);
    } else {
#pragma unroll
        for (int c = 0; c < N; c += 8) tmem_ld8(taddr + c, v + c);
    }
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Wait for phase `parity` with a bound of about one second; gives up early
// when another role of the block raised *abort.  On a timeout it raises
// *abort and records SHS_ERR_TIMEOUT in *status.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort,
                                                   int* status) {
    const uint64_t t0 = now_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 63u) {
            if (*abort) return false;
            if (now_ns() - t0 > 1000000000ull) {
                *abort = 1;
                atomicExch(status, 5);
                return false;
            }
        }
    }
}

}  // namespace tc
}  // namespace shs
