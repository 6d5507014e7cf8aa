// Reduced-precision tails of the 8-band path on the fifth-generation tensor
// cores (tcgen05): the SH exponential's squarings (Eq. 7, truncated) and the
// shading (Eq. 8), forward and adjoint.  Compiled once with -DSHS_NB=8.
//
// Squaring through an exact quadrature.  The product of three SH expansions
// of fewer than 8 bands is a polynomial of degree <= 21 on the sphere, so the
// rule of 11 Gauss-Legendre nodes in z times 22 uniform azimuths (242
// directions w_q, padded to 256 with zero weight) integrates it exactly:
//   (S * S)_j = sum_q w_q S(w_q)^2 y_j(w_q).
// For a tile of 128 points (one tensor-memory lane each) a squaring is two
// GEMMs: X = S Y^T (values at the directions) and S' = (X o X) (w Y).  The
// directions are taken in chunks of CQ; the tables Y_c and (2^8 w Y)_c of a
// chunk are streamed from global memory (L2-resident) through a ring of
// shared-memory stages by bulk copies.
//
// Shading through the same rule.  B_c = a_c int L_c V H = a_c e0 sum_q w_q
// X_S(w_q) H(n . w_q) L_c(w_q) with X_S = S Y^T after the last squaring and
// H(t) = sum_l A_l (2l+1)/(4 pi) P_l(t) the clamped-cosine lobe (addition
// theorem), an even polynomial in t plus A_1 3/(4 pi) t (A_l = 0 for odd
// l >= 3).  X_S comes from the tensor cores; the sum over directions runs on
// the CUDA cores.
//
// Roles in a block of 160 threads: warps 0-3 are the compute warps (thread
// = point = tensor-memory lane): exponent set-up, squaring and splitting the
// GEMM outputs, the direction sums.  Lane 0 of warp 4 issues the MMAs and the
// table copies.  Hand-offs go through mbarriers; every wait is bounded (about
// one second) and a timeout makes every role stop, drain its copies and MMAs
// and return with SHS_ERR_TIMEOUT in the status word.

#include <cstdint>
#include <cuda_runtime.h>

#include "generated/shs_sh_gen.cuh"
#include "shs_internal.h"
#include "shs_exp.cuh"
#include "shs_tc.cuh"
#include "shs_warp.cuh"

#if SHS_NB != 8
#error "the tensor-core tails are compiled for 8 bands only"
#endif

namespace shs {
namespace {

constexpr int K = 64;
constexpr int KPAD = 64;
constexpr int kQ = kTcQ;          // 256 directions (242 with weight)
constexpr int kCompute = 128;     // compute threads
constexpr int kThreads = 160;     // + the MMA / copy warp
constexpr int kSmemBudget = 227 * 1024;
using SH = shsgen::SH<8>;

// Shared-memory plan of one tail kernel: per-point split operands (A: S, and
// for the adjoint A2: dS), double-buffered chunk operands Xs, the table ring,
// and the direction table.
template <int PR, int CQ, bool BWD>
struct Plan {
    using P = tc::Prec<PR>;
    static constexpr int EB = P::kElem, NP = P::kParts;
    static constexpr int NCH = kQ / CQ;
    static constexpr uint32_t kA = 128u * 64 * EB;      // one part of a [128 x 64] operand
    static constexpr uint32_t kXs = 128u * CQ * EB;     // one part of a [128 x CQ] operand
    static constexpr uint32_t kTb = CQ * 64u * EB;      // one part of Y_c or (wY)_c
    static constexpr uint32_t kChunk = 2u * NP * kTb;   // Y_c parts, then (wY)_c parts
    static constexpr uint32_t kOffA = 0;
    static constexpr uint32_t kOffA2 = kOffA + NP * kA;
    static constexpr uint32_t kOffXs = kOffA2 + (BWD ? NP * kA : 0);
    static constexpr uint32_t kOffDir = kOffXs + 2 * NP * kXs;
    static constexpr uint32_t kOffRing = kOffDir + kQ * 28;   // float4 dir, 3 floats of light
    static constexpr int kStatic = 4096;                       // barriers, flags, per-warp sums
    static constexpr int R0 = static_cast<int>((kSmemBudget - kStatic - kOffRing) / kChunk);
    static constexpr int R = R0 > 4 ? 4 : R0;
    static_assert(R >= 2, "table ring needs two stages");
    static constexpr uint32_t kBytes = kOffRing + R * kChunk;
    static constexpr uint32_t kIdescX = tc::idesc_of<PR>(128, CQ);   // X_c = A Y_c^T
    static constexpr uint32_t kIdescS = tc::idesc_of<PR>(128, 64);   // S' += Xs (wY)_c
};

// Lobe H(t) = c1 t + e0 + e1 t^2 + e2 t^4 + e3 t^6 and its derivative.
struct Lobe {
    float c1, e0, e1, e2, e3;
};
__device__ __forceinline__ float lobe(const Lobe& h, float t) {
    const float u = t * t;
    return fmaf(h.c1, t, fmaf(fmaf(fmaf(h.e3, u, h.e2), u, h.e1), u, h.e0));
}
__device__ __forceinline__ float lobe_d(const Lobe& h, float t) {
    const float u = t * t;
    return fmaf(t * fmaf(fmaf(6.f * h.e3, u, 4.f * h.e2), u, 2.f * h.e1), 1.f, h.c1);
}

// Row scaling by a power of two keeps half-precision operands and their
// squares in range and clear of underflow: sum |S| 2^-s in [2^5, 2^6) bounds
// |X| by 2^7 (|y_i| <= 1.1).
__device__ __forceinline__ int row_shift(const float* S) {
    float sabs = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) sabs += fabsf(S[i]);
    if (!(sabs > 1e-30f)) return 0;
    return min(64, max(-64, ilogbf(1.25f * sabs) - 6));
}

template <int PR>
__device__ __forceinline__ void store_operand64(unsigned char* base, uint32_t part_bytes, int row, const float* S,
                                                int sh) {
    float Sd[K];
#pragma unroll
    for (int i = 0; i < K; ++i) Sd[i] = ldexpf(S[i], -sh);
    tc::store_row_split<PR, 64>(base, part_bytes, row, Sd);
}

// Direction table: s_dir[q] = (x, y, z, w_q), s_lc[c][q] = L_c(w_q).
__device__ void load_directions(const TcArgs& a, float4* s_dir, float (*s_lc)[kQ]) {
    for (int q = threadIdx.x; q < kQ; q += kCompute) {
        s_dir[q] = __ldg(a.dirs + q);
        const float* y = a.ytab + q * K;
        float l0 = 0.f, l1 = 0.f, l2 = 0.f;
#pragma unroll 8
        for (int i = 0; i < K; ++i) {
            const float yi = __ldg(y + i);
            l0 = fmaf(__ldg(a.sc.light + i), yi, l0);
            l1 = fmaf(__ldg(a.sc.light + KPAD + i), yi, l1);
            l2 = fmaf(__ldg(a.sc.light + 2 * KPAD + i), yi, l2);
        }
        s_lc[0][q] = l0;
        s_lc[1][q] = l1;
        s_lc[2][q] = l2;
    }
}

// A compute warp's wait: the outcome is made uniform over the warp so that its
// lanes leave together (they run warp-wide shuffles later).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* status) {
    return __all_sync(0xffffffffu, tc::mbar_wait_or_abort(bar, parity, abort, status));
}

__device__ __forceinline__ void named_sync_compute() {
    asm volatile("bar.sync 1, 128;" ::: "memory");
}

// Exponent set-up of one point (DC isolation, scaling, optimal linear step):
// S_0 and k, e0.
struct ExpState {
    int k;
    float e0, scale, nrm2;
    OLCoef ol;
};
__device__ __forceinline__ ExpState exp_setup(const SceneView& sc, const float* f, float* S) {
    ExpState x;
    x.nrm2 = 0.f;
#pragma unroll
    for (int i = 1; i < K; ++i) x.nrm2 = fmaf(f[i], f[i], x.nrm2);
    x.k = scaling_k(sc, x.nrm2);
    x.e0 = expf(f[0] * kInvSqrt4Pi);
    x.scale = ldexpf(1.f, -x.k);
    x.ol = ol_coef(sc, x.nrm2 * x.scale * x.scale);
    S[0] = x.ol.a * kSqrt4Pi;
#pragma unroll
    for (int i = 1; i < K; ++i) S[i] = x.ol.b * (f[i] * x.scale);
    return x;
}

// ---------------------------------------------------------------------------
// MMA / copy role (one thread)
// ---------------------------------------------------------------------------
// Chunk sequence: every pass over the directions consumes chunks 0..NCH-1 in
// order; the global count `seq` numbers them, stage = seq % R.  The issuer
// keeps copies R - 2 chunks ahead: at step seq it refills the stage of chunk
// seq - 2 (whose MMAs it committed a step earlier) with chunk seq - 2 + R.
template <int R, int NCH, uint32_t CHUNK>
struct Ring {
    uint64_t* full;
    uint64_t* empty;
    unsigned char* base;
    const unsigned char* src;
    uint32_t issued = 0;

    __device__ void load(uint32_t s) {
        const uint32_t st = s % R;
        tc::mbar_expect(&full[st], CHUNK);
        tc::bulk_g2s(base + st * CHUNK, src + static_cast<size_t>(s % NCH) * CHUNK, CHUNK, &full[st]);
    }
    __device__ void prime() {
        for (uint32_t s = 0; s < static_cast<uint32_t>(R); ++s) load(s);
        issued = R;
    }
    // Load chunk `issued` into the stage of chunk issued - R once that
    // chunk's MMAs have completed.
    __device__ bool load_next(volatile int* abort, int* status) {
        if (issued >= static_cast<uint32_t>(R)) {
            const uint32_t old = issued - R;
            if (!tc::mbar_wait_or_abort(&empty[old % R], (old / R) & 1u, abort, status)) return false;
        }
        load(issued);
        ++issued;
        return true;
    }
    // Before consuming chunk seq: make sure its copy was issued.
    __device__ bool ensure(uint32_t seq, volatile int* abort, int* status) {
        while (issued <= seq)
            if (!load_next(abort, status)) return false;
        return true;
    }
    // After step seq committed the release of chunk seq - 1: refill the stage
    // released a step earlier (chunk seq - 2), if not done yet.
    __device__ bool refill(uint32_t seq, volatile int* abort, int* status) {
        if (seq < 2 || issued > seq - 2 + R) return true;
        return load_next(abort, status);
    }
    __device__ unsigned char* stage(uint32_t s) const { return base + (s % R) * CHUNK; }
    // Wait (bounded, ignoring aborts) for every copy still in flight.
    __device__ void drain(uint32_t consumed) {
        for (uint32_t s = consumed; s < issued; ++s) (void)tc::mbar_wait(&full[s % R], (s / R) & 1u);
    }
};

// ---------------------------------------------------------------------------
// forward tail
// ---------------------------------------------------------------------------
template <int PR, int CQ>
__global__ void __launch_bounds__(kThreads, 1) tail_fwd_tc_kernel(const __grid_constant__ TcArgs a) {
    using PL = Plan<PR, CQ, false>;
    constexpr int NCH = PL::NCH, R = PL::R;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[R], empty[R], xr[2], xs[2], g2[2], ar, sp, fin;
    __shared__ uint32_t tmem_base;
    __shared__ int s_kt;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char* sA = sm + PL::kOffA;
    unsigned char* sXs = sm + PL::kOffXs;
    float4* s_dir = reinterpret_cast<float4*>(sm + PL::kOffDir);
    float (*s_lc)[kQ] = reinterpret_cast<float (*)[kQ]>(s_dir + kQ);
    unsigned char* sRing = sm + PL::kOffRing;
    volatile int* abort = &s_abort;

    if (warp == 0) tc::tmem_alloc(&tmem_base, 128);
    if (tid == 0) {
        for (int i = 0; i < R; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&xr[i], 1);
            tc::mbar_init(&xs[i], kCompute);
            tc::mbar_init(&g2[i], 1);
        }
        tc::mbar_init(&ar, kCompute);
        tc::mbar_init(&sp, 1);
        tc::mbar_init(&fin, 1);
        s_kt = 0;
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const int64_t P = a.n_points;
    const int64_t ntiles = (P + 127) / 128;

    if (warp == 4) {
        if ((tid & 31) == 0) {
            // ---------------- MMA / copy issuer
            Ring<R, NCH, PL::kChunk> ring{full, empty, sRing, static_cast<const unsigned char*>(a.chunks)};
            ring.prime();
            uint32_t seq = 0, arc = 0, xsc[2] = {0u, 0u};
            bool ok = true;
            const uint32_t aA = tc::smem_u32(sA), aXs = tc::smem_u32(sXs);
            for (int64_t tile = blockIdx.x, it = 0; ok && tile < ntiles; tile += gridDim.x, ++it) {
                int kt = 0;
                for (int pass = 0; ok; ++pass) {
                    ok = tc::mbar_wait_or_abort(&ar, arc & 1u, abort, a.sc.status);
                    ++arc;
                    if (!ok) break;
                    tc::fence_after_sync();
                    if (pass == 0) kt = s_kt & 31;
                    const bool shading = pass == kt;
                    for (int c = 0; ok && c < NCH; ++c, ++seq) {
                        ok = ring.ensure(seq, abort, a.sc.status) &&
                             tc::mbar_wait_or_abort(&full[seq % R], (seq / R) & 1u, abort, a.sc.status);
                        if (!ok) break;
                        const uint32_t st = tc::smem_u32(ring.stage(seq));
                        tc::gemm_split<PR, 64>(tmem + (c & 1) * 32, aA, PL::kA, st, PL::kTb, PL::kIdescX, false);
                        tc::commit(&xr[c & 1]);
                        if (c >= 1) {
                            const int b = (c - 1) & 1;
                            ok = tc::mbar_wait_or_abort(&xs[b], xsc[b] & 1u, abort, a.sc.status);
                            ++xsc[b];
                            if (!ok) break;
                            tc::fence_after_sync();
                            if (!shading) {
                                const uint32_t stp = tc::smem_u32(ring.stage(seq - 1));
                                tc::gemm_split<PR, CQ>(tmem + 64, aXs + b * PL::NP * PL::kXs, PL::kXs,
                                                       stp + PL::NP * PL::kTb, PL::kTb, PL::kIdescS, c - 1 > 0);
                                tc::commit(&g2[b]);
                            }
                            tc::commit(&empty[(seq - 1) % R]);
                        }
                        ok = ring.refill(seq, abort, a.sc.status);
                    }
                    if (!ok) break;
                    // last chunk of the pass
                    const int b = (NCH - 1) & 1;
                    ok = tc::mbar_wait_or_abort(&xs[b], xsc[b] & 1u, abort, a.sc.status);
                    ++xsc[b];
                    if (!ok) break;
                    tc::fence_after_sync();
                    if (!shading) {
                        const uint32_t stp = tc::smem_u32(ring.stage(seq - 1));
                        tc::gemm_split<PR, CQ>(tmem + 64, aXs + b * PL::NP * PL::kXs, PL::kXs,
                                               stp + PL::NP * PL::kTb, PL::kTb, PL::kIdescS, NCH > 1);
                        tc::commit(&g2[b]);
                    }
                    tc::commit(&empty[(seq - 1) % R]);
                    if (!shading) tc::commit(&sp);
                    if (shading) break;
                }
            }
            ring.drain(seq);
            tc::commit(&fin);
            (void)tc::mbar_wait(&fin, 0);
        }
    } else {
        // ---------------- compute warps
        load_directions(a, s_dir, s_lc);
        named_sync_compute();
        const uint32_t lane_tm = tmem + (static_cast<uint32_t>(warp * 32) << 16);
        const Lobe hl{a.lobe_c1, a.lobe_e[0], a.lobe_e[1], a.lobe_e[2], a.lobe_e[3]};
        uint32_t xrc[2] = {0u, 0u}, g2c[2] = {0u, 0u}, spc = 0, arc = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x, it = 0; ok && tile < ntiles; tile += gridDim.x, ++it) {
            const int64_t p = tile * 128 + tid;
            const bool live = p < P;
            const int64_t q = live ? p : 0;
            float S[K];
#pragma unroll
            for (int i = 0; i < K; ++i) S[i] = live ? __ldg(a.f + i * P + q) : 0.f;
            const ExpState ex = exp_setup(a.sc, S, S);
            atomicMax(&s_kt, static_cast<int>((it << 5) | ex.k));
            float ux = 0.f, uy = 0.f, uz = 1.f;
            if (live) {
                const float nx = __ldg(a.normals + 3 * q), ny = __ldg(a.normals + 3 * q + 1),
                            nz = __ldg(a.normals + 3 * q + 2);
                const float n2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
                const float il = n2 > 0.f ? rsqrtf(n2) : 0.f;
                ux = nx * il;
                uy = ny * il;
                uz = nz * il;
            }
            float B0 = 0.f, B1 = 0.f, B2 = 0.f;
            int kt = 0, sh = 0;
            for (int pass = 0; ok; ++pass) {
                sh = row_shift(S);
                store_operand64<PR>(sA, PL::kA, tid, S, sh);
                tc::fence_async_smem();
                tc::fence_before_sync();
                tc::mbar_arrive(&ar);
                if (pass == 0) {
                    ok = warp_wait(&ar, arc & 1u, abort, a.sc.status);
                    if (!ok) break;
                    kt = s_kt & 31;
                }
                ++arc;
                const bool shading = pass == kt;
                for (int c = 0; ok && c < NCH; ++c) {
                    const int b = c & 1;
                    ok = warp_wait(&xr[b], xrc[b] & 1u, abort, a.sc.status);
                    ++xrc[b];
                    if (!ok) break;
                    tc::fence_after_sync();
                    float X[CQ];
                    tc::tmem_ld<CQ>(lane_tm + b * 32, X);
                    if (!shading) {
#pragma unroll
                        for (int i = 0; i < CQ; ++i) X[i] *= X[i];
                        if (c >= 2) {
                            ok = warp_wait(&g2[b], (g2c[b] - 1) & 1u, abort, a.sc.status);
                            if (!ok) break;
                        }
                        tc::store_row_split<PR, CQ>(sXs + b * PL::NP * PL::kXs, PL::kXs, tid, X);
                        tc::fence_async_smem();
                        tc::fence_before_sync();
                        tc::mbar_arrive(&xs[b]);
                        ++g2c[b];
                    } else {
#pragma unroll 4
                        for (int i = 0; i < CQ; ++i) {
                            const int qd = c * CQ + i;
                            const float4 d = s_dir[qd];
                            const float t = fmaf(ux, d.x, fmaf(uy, d.y, uz * d.z));
                            const float xw = X[i] * lobe(hl, t) * d.w;
                            B0 = fmaf(xw, s_lc[0][qd], B0);
                            B1 = fmaf(xw, s_lc[1][qd], B1);
                            B2 = fmaf(xw, s_lc[2][qd], B2);
                        }
                        tc::fence_before_sync();
                        tc::mbar_arrive(&xs[b]);
                    }
                }
                if (!ok || shading) break;
                ok = warp_wait(&sp, spc & 1u, abort, a.sc.status);
                ++spc;
                if (!ok) break;
                tc::fence_after_sync();
                float Sn[K];
                tc::tmem_ld<64>(lane_tm + 64, Sn);
                tc::fence_before_sync();
                if (pass < ex.k) {
                    const float up = ldexpf(a.b2_unscale, 2 * sh);
#pragma unroll
                    for (int i = 0; i < K; ++i) S[i] = Sn[i] * up;
                }
            }
            if (!ok) break;
            if (live) {
                const float s3 = ex.e0 * ldexpf(1.f, sh);
                a.radiance[3 * q] = __ldg(a.albedo + 3 * q) * B0 * s3;
                a.radiance[3 * q + 1] = __ldg(a.albedo + 3 * q + 1) * B1 * s3;
                a.radiance[3 * q + 2] = __ldg(a.albedo + 3 * q + 2) * B2 * s3;
                if (a.saved_k) a.saved_k[q] = ex.k;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------------------
// adjoint tail
// ---------------------------------------------------------------------------
// Per tile, 2 kt + 1 passes over the directions (kt = the tile's largest k):
//   passes 0..kt-1  recompute the squarings S_{t+1} = S_t * S_t as in the
//                   forward, keeping each operand S_t (float32) in a per-block
//                   workspace;
//   pass kt         shading adjoint from X_S = S_k Y^T: with u_c = a_c dB_c and
//                   D(w) = sum_c u_c L_c(w), the direction sums give
//                   dB_c/da_c, dL/de0 = int D H V / e0 and dL/dn = e0 int D V
//                   H'(n.w) w (projected, through n/|n|); two GEMMs project
//                   dV = P[D H] and W = V * H = e0 P[X_S H] (d_light = sum over
//                   points of u_c W);
//   passes kt+1..2kt  the squarings' adjoint, t = kt-1 down to 0:
//                   dS_t = 2 P[(S_t Y^T) o (dS_{t+1} Y^T)], three GEMMs per
//                   chunk (the tables are those of the forward: the adjoint of
//                   projecting with w Y is evaluating with Y, and back).
// Then the optimal-linear step and the scaling in float32 (as the CUDA-core
// adjoint) give df, stored for the pair pass.
template <int PR, int CQ>
__global__ void __launch_bounds__(kThreads, 1) tail_bwd_tc_kernel(const __grid_constant__ TcArgs a) {
    using PL = Plan<PR, CQ, true>;
    constexpr int NCH = PL::NCH, R = PL::R, NP = PL::NP;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[R], empty[R], xr[2], xs[2], g2[2], ar, sp, fin;
    __shared__ uint32_t tmem_base;
    __shared__ int s_kt;
    __shared__ int s_abort;
    __shared__ float s_dl[4][3 * K + 1];
    __shared__ float s_lsum[3];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* sA = sm + PL::kOffA;
    unsigned char* sA2 = sm + PL::kOffA2;
    unsigned char* sXs = sm + PL::kOffXs;
    float4* s_dir = reinterpret_cast<float4*>(sm + PL::kOffDir);
    float (*s_lc)[kQ] = reinterpret_cast<float (*)[kQ]>(s_dir + kQ);
    unsigned char* sRing = sm + PL::kOffRing;
    volatile int* abort = &s_abort;

    if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
    if (tid == 0) {
        for (int i = 0; i < R; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&xr[i], 1);
            tc::mbar_init(&xs[i], kCompute);
            tc::mbar_init(&g2[i], 1);
        }
        tc::mbar_init(&ar, kCompute);
        tc::mbar_init(&sp, 1);
        tc::mbar_init(&fin, 1);
        s_kt = 0;
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < 4 * (3 * K + 1); e += kThreads) (&s_dl[0][0])[e] = 0.f;
    if (tid < 3) {
        float t = 0.f;
        for (int i = 0; i < K; ++i) t += fabsf(__ldg(a.sc.light + tid * KPAD + i));
        s_lsum[tid] = t;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const int64_t P = a.n_points;
    const int64_t ntiles = (P + 127) / 128;

    if (warp == 4) {
        if (lane == 0) {
            // ---------------- MMA / copy issuer
            Ring<R, NCH, PL::kChunk> ring{full, empty, sRing, static_cast<const unsigned char*>(a.chunks)};
            ring.prime();
            uint32_t seq = 0, arc = 0, xsc[2] = {0u, 0u};
            bool ok = true;
            const uint32_t aA = tc::smem_u32(sA), aA2 = tc::smem_u32(sA2), aXs = tc::smem_u32(sXs);
            for (int64_t tile = blockIdx.x, it = 0; ok && tile < ntiles; tile += gridDim.x, ++it) {
                int kt = 0;
                for (int pass = 0; ok && pass <= 2 * kt; ++pass) {
                    ok = tc::mbar_wait_or_abort(&ar, arc & 1u, abort, a.sc.status);
                    ++arc;
                    if (!ok) break;
                    tc::fence_after_sync();
                    if (pass == 0) kt = s_kt & 31;
                    const bool shade = pass == kt, adj = pass > kt;
                    for (int c = 0; ok && c <= NCH; ++c) {
                        if (c < NCH) {
                            ok = ring.ensure(seq, abort, a.sc.status) &&
                                 tc::mbar_wait_or_abort(&full[seq % R], (seq / R) & 1u, abort, a.sc.status);
                            if (!ok) break;
                            const uint32_t st = tc::smem_u32(ring.stage(seq));
                            tc::gemm_split<PR, 64>(tmem + (c & 1) * 32, aA, PL::kA, st, PL::kTb, PL::kIdescX, false);
                            if (adj)
                                tc::gemm_split<PR, 64>(tmem + 64 + (c & 1) * 32, aA2, PL::kA, st, PL::kTb, PL::kIdescX,
                                                       false);
                            tc::commit(&xr[c & 1]);
                        }
                        if (c >= 1) {
                            const int b = (c - 1) & 1;
                            ok = tc::mbar_wait_or_abort(&xs[b], xsc[b] & 1u, abort, a.sc.status);
                            ++xsc[b];
                            if (!ok) break;
                            tc::fence_after_sync();
                            const uint32_t wy = tc::smem_u32(ring.stage(seq - 1)) + NP * PL::kTb;
                            tc::gemm_split<PR, CQ>(tmem + 128, aXs + b * NP * PL::kXs, PL::kXs, wy, PL::kTb,
                                                   PL::kIdescS, c - 1 > 0);
                            if (shade)
                                tc::gemm_split<PR, CQ>(tmem + 192, aA2 + b * NP * PL::kXs, PL::kXs, wy, PL::kTb,
                                                       PL::kIdescS, c - 1 > 0);
                            tc::commit(&g2[b]);
                            tc::commit(&empty[(seq - 1) % R]);
                            if (c == NCH) tc::commit(&sp);
                        }
                        if (c < NCH) {
                            ok = ring.refill(seq, abort, a.sc.status);
                            ++seq;
                        }
                    }
                }
            }
            ring.drain(seq);
            tc::commit(&fin);
            (void)tc::mbar_wait(&fin, 0);
        }
    } else {
        // ---------------- compute warps
        load_directions(a, s_dir, s_lc);
        named_sync_compute();
        const uint32_t lane_tm = tmem + (static_cast<uint32_t>(warp * 32) << 16);
        const Lobe hl{a.lobe_c1, a.lobe_e[0], a.lobe_e[1], a.lobe_e[2], a.lobe_e[3]};
        float* hist = a.hist + static_cast<size_t>(blockIdx.x) * (kMaxK * K * 128);
        uint32_t xrc[2] = {0u, 0u}, g2c[2] = {0u, 0u}, spc = 0, arc = 0;
        float loss_acc = 0.f;
        bool ok = true;
        for (int64_t tile = blockIdx.x, it = 0; ok && tile < ntiles; tile += gridDim.x, ++it) {
            const int64_t p = tile * 128 + tid;
            const bool live = p < P;
            const int64_t q = live ? p : 0;
            float V[K];      // S (forward passes), then dS (adjoint passes)
#pragma unroll
            for (int i = 0; i < K; ++i) V[i] = live ? __ldg(a.f + i * P + q) : 0.f;
            float nrm2 = 0.f;
#pragma unroll
            for (int i = 1; i < K; ++i) nrm2 = fmaf(V[i], V[i], nrm2);
            const int k = a.k_in ? (live ? min(max(__ldg(a.k_in + q), 0), kMaxK) : 0) : scaling_k(a.sc, nrm2);
            const float e0 = expf(V[0] * kInvSqrt4Pi);
            const float scale = ldexpf(1.f, -k);
            const OLCoef ol = ol_coef(a.sc, nrm2 * scale * scale);
            V[0] = ol.a * kSqrt4Pi;
#pragma unroll
            for (int i = 1; i < K; ++i) V[i] = ol.b * (V[i] * scale);
            atomicMax(&s_kt, static_cast<int>((it << 5) | k));
            float ux = 0.f, uy = 0.f, uz = 1.f, il = 0.f;
            float dB[3] = {0.f, 0.f, 0.f}, u[3] = {0.f, 0.f, 0.f}, alb[3] = {0.f, 0.f, 0.f};
            if (live) {
                const float nx = __ldg(a.normals + 3 * q), ny = __ldg(a.normals + 3 * q + 1),
                            nz = __ldg(a.normals + 3 * q + 2);
                const float n2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
                il = n2 > 0.f ? rsqrtf(n2) : 0.f;
                ux = nx * il;
                uy = ny * il;
                uz = nz * il;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    alb[c] = __ldg(a.albedo + 3 * q + c);
                    if (a.target) {
                        dB[c] = __ldg(a.radiance_in + 3 * q + c) - __ldg(a.target + 3 * q + c);
                        loss_acc = fmaf(0.5f * dB[c], dB[c], loss_acc);
                    } else {
                        dB[c] = __ldg(a.d_radiance + 3 * q + c);
                    }
                    u[c] = alb[c] * dB[c];
                }
            }
            // scale of D H (the shading adjoint's projected operand): |L_c(w)| <= 1.1 sum |L_c,i|, |H| <= 1.1
            const int sz = [&] {
                const float zb = 1.25f * (fabsf(u[0]) * s_lsum[0] + fabsf(u[1]) * s_lsum[1] + fabsf(u[2]) * s_lsum[2]);
                return zb > 1e-30f ? min(64, max(-64, ilogbf(zb) - 6)) : 0;
            }();
            float acc[3] = {0.f, 0.f, 0.f}, gn[3] = {0.f, 0.f, 0.f}, de0s = 0.f;
            float de0 = 0.f;
            int kt = 0, sh = 0, shg = 0;
            for (int pass = 0; ok && pass <= 2 * kt; ++pass) {
                // operands of this pass (kt is still 0 before pass 0's barrier)
                if (pass <= kt) {
                    // forward passes and the shading pass: A = S_pass
                    sh = row_shift(V);
                    store_operand64<PR>(sA, PL::kA, tid, V, sh);
                    if (pass == 0 || pass < kt) {
                        // keep S_t for the adjoint (read back for t < kt only)
#pragma unroll 8
                        for (int i = 0; i < K; ++i) hist[(static_cast<size_t>(pass) * K + i) * 128 + tid] = V[i];
                    }
                } else {
                    const int t = 2 * kt - pass;
                    float Sh[K];
#pragma unroll 8
                    for (int i = 0; i < K; ++i) Sh[i] = hist[(static_cast<size_t>(t) * K + i) * 128 + tid];
                    sh = row_shift(Sh);
                    store_operand64<PR>(sA, PL::kA, tid, Sh, sh);
                    shg = row_shift(V);
                    store_operand64<PR>(sA2, PL::kA, tid, V, shg);
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
                tc::mbar_arrive(&ar);
                if (pass == 0) {
                    ok = warp_wait(&ar, arc & 1u, abort, a.sc.status);
                    if (!ok) break;
                    kt = s_kt & 31;
                }
                ++arc;
                const bool shade = pass == kt, adj = pass > kt;
                for (int c = 0; ok && c < NCH; ++c) {
                    const int b = c & 1;
                    ok = warp_wait(&xr[b], xrc[b] & 1u, abort, a.sc.status);
                    ++xrc[b];
                    if (!ok) break;
                    tc::fence_after_sync();
                    float X[CQ];
                    tc::tmem_ld<CQ>(lane_tm + b * 32, X);
                    if (adj) {
                        float G[CQ];
                        tc::tmem_ld<CQ>(lane_tm + 64 + b * 32, G);
#pragma unroll
                        for (int i = 0; i < CQ; ++i) X[i] = 2.f * X[i] * G[i];
                    } else if (!shade) {
#pragma unroll
                        for (int i = 0; i < CQ; ++i) X[i] *= X[i];
                    } else {
                        float Z[CQ];
#pragma unroll 4
                        for (int i = 0; i < CQ; ++i) {
                            const int qd = c * CQ + i;
                            const float4 d = s_dir[qd];
                            const float4 l = make_float4(s_lc[0][qd], s_lc[1][qd], s_lc[2][qd], 0.f);
                            const float t = fmaf(ux, d.x, fmaf(uy, d.y, uz * d.z));
                            const float h = lobe(hl, t), hd = lobe_d(hl, t);
                            const float D = fmaf(u[0], l.x, fmaf(u[1], l.y, u[2] * l.z));
                            const float wx = d.w * X[i];
                            const float wxh = wx * h;
                            acc[0] = fmaf(wxh, l.x, acc[0]);
                            acc[1] = fmaf(wxh, l.y, acc[1]);
                            acc[2] = fmaf(wxh, l.z, acc[2]);
                            de0s = fmaf(wxh, D, de0s);
                            const float gd = wx * D * hd;
                            gn[0] = fmaf(gd, d.x, gn[0]);
                            gn[1] = fmaf(gd, d.y, gn[1]);
                            gn[2] = fmaf(gd, d.z, gn[2]);
                            Z[i] = ldexpf(D * h, -sz);
                            X[i] *= h;
                        }
                        if (c >= 2) {
                            ok = warp_wait(&g2[b], (g2c[b] - 1) & 1u, abort, a.sc.status);
                            if (!ok) break;
                        }
                        tc::store_row_split<PR, CQ>(sXs + b * NP * PL::kXs, PL::kXs, tid, Z);
                        tc::store_row_split<PR, CQ>(sA2 + b * NP * PL::kXs, PL::kXs, tid, X);
                        tc::fence_async_smem();
                        tc::fence_before_sync();
                        tc::mbar_arrive(&xs[b]);
                        ++g2c[b];
                        continue;
                    }
                    if (c >= 2) {
                        ok = warp_wait(&g2[b], (g2c[b] - 1) & 1u, abort, a.sc.status);
                        if (!ok) break;
                    }
                    tc::store_row_split<PR, CQ>(sXs + b * NP * PL::kXs, PL::kXs, tid, X);
                    tc::fence_async_smem();
                    tc::fence_before_sync();
                    tc::mbar_arrive(&xs[b]);
                    ++g2c[b];
                }
                if (!ok) break;
                ok = warp_wait(&sp, spc & 1u, abort, a.sc.status);
                ++spc;
                if (!ok) break;
                tc::fence_after_sync();
                float Sn[K];
                tc::tmem_ld<64>(lane_tm + 128, Sn);
                if (pass < kt) {
                    tc::fence_before_sync();
                    if (pass < k) {
                        const float up = ldexpf(a.b2_unscale, 2 * sh);
#pragma unroll
                        for (int i = 0; i < K; ++i) V[i] = Sn[i] * up;
                    }
                } else if (shade) {
                    // dS_k = e0 dV, W = e0 2^sh P[X H]; d_light += u_c W over the points
                    float Wv[K];
                    tc::tmem_ld<64>(lane_tm + 192, Wv);
                    tc::fence_before_sync();
                    const float dvs = e0 * ldexpf(a.b2_unscale, sz);
#pragma unroll
                    for (int i = 0; i < K; ++i) V[i] = Sn[i] * dvs;
                    const float ws = e0 * ldexpf(a.b2_unscale, sh);
#pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        float dl[K];
                        const float uc = live ? u[c3] * ws : 0.f;
#pragma unroll
                        for (int i = 0; i < K; ++i) dl[i] = uc * Wv[i];
                        warp_sum_into<K>(dl, &s_dl[warp][c3 * K], lane);
                    }
                    const float s2 = ldexpf(1.f, sh);
                    de0 = de0s * s2;
                    if (live) {
                        if (a.d_albedo) {
#pragma unroll
                            for (int c3 = 0; c3 < 3; ++c3) a.d_albedo[3 * q + c3] = dB[c3] * e0 * s2 * acc[c3];
                        }
                        if (a.d_normals) {
                            const float gx = e0 * s2 * gn[0], gy = e0 * s2 * gn[1], gz = e0 * s2 * gn[2];
                            const float ug = ux * gx + uy * gy + uz * gz;
                            a.d_normals[3 * q] = (gx - ux * ug) * il;
                            a.d_normals[3 * q + 1] = (gy - uy * ug) * il;
                            a.d_normals[3 * q + 2] = (gz - uz * ug) * il;
                        }
                    }
                } else {
                    tc::fence_before_sync();
                    if (2 * kt - pass < k) {
                        const float up = ldexpf(a.b2_unscale, sh + shg);
#pragma unroll
                        for (int i = 0; i < K; ++i) V[i] = Sn[i] * up;
                    }
                }
            }
            if (!ok) break;
            // optimal linear step and scaling: S_0 = a(s) sqrt(4 pi), S_i = b(s) g_i, g = f^ 2^-k
            if (live) {
                float dBs = 0.f;
#pragma unroll
                for (int i = 1; i < K; ++i) dBs = fmaf(V[i], __ldg(a.f + i * P + q) * scale, dBs);
                const float dA = V[0] * kSqrt4Pi;
                const float cg = fmaf(dA, ol.ca, dBs * ol.cb);
                a.dfp_ws[q] = de0 * e0 * kInvSqrt4Pi * a.sc.neg_2pi_eps * SH::norm(0);
#pragma unroll
                for (int i = 1; i < K; ++i) {
                    const float gi = __ldg(a.f + i * P + q) * scale;
                    a.dfp_ws[i * P + q] = fmaf(ol.b, V[i], cg * gi) * scale * a.sc.neg_2pi_eps * SH::norm(i);
                }
            }
        }
        if (a.target) {
            const float v = warp_sum(loss_acc);
            if (lane == 0) s_dl[warp][3 * K] += v;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
    if (s_abort) return;
    // block partial row of the lighting gradient and loss
    for (int e = tid; e <= 3 * K; e += kThreads) {
        const float v = s_dl[0][e] + s_dl[1][e] + s_dl[2][e] + s_dl[3][e];
        if (a.deterministic) {
            a.partials[static_cast<size_t>(blockIdx.x) * a.partial_stride + e] = v;
            for (int r = blockIdx.x + gridDim.x; r < a.partial_rows; r += gridDim.x)
                a.partials[static_cast<size_t>(r) * a.partial_stride + e] = 0.f;
        } else {
            atomicAdd(a.partials + e, v);
        }
    }
}

template <int PR, int CQ>
cudaError_t launch_fwd_t(const TcArgs& a, cudaStream_t s) {
    using PL = Plan<PR, CQ, false>;
    auto kern = tail_fwd_tc_kernel<PR, CQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(PL::kBytes));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (a.n_points + 127) / 128;
    const int grid = static_cast<int>(tiles < sms ? tiles : sms);
    kern<<<grid, kThreads, PL::kBytes, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <int PR, int CQ>
cudaError_t launch_bwd_t(const TcArgs& a, cudaStream_t s) {
    using PL = Plan<PR, CQ, true>;
    auto kern = tail_bwd_tc_kernel<PR, CQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(PL::kBytes));
    if (e != cudaSuccess) return e;
    const int64_t tiles = (a.n_points + 127) / 128;
    const int cap = tail_tc_bwd_grid();
    const int grid = static_cast<int>(tiles < cap ? tiles : cap);
    kern<<<grid, kThreads, PL::kBytes, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

int tail_tc_bwd_grid() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return sms > 0 ? sms : 1;
}

cudaError_t launch_tail_tc_bwd(const TcArgs& a, cudaStream_t s) {
    if (a.n_points <= 0) return cudaSuccess;
    switch (a.prec) {
        case tc::kPrecBF16: return launch_bwd_t<tc::kPrecBF16, 32>(a, s);
        case tc::kPrecFP16: return launch_bwd_t<tc::kPrecFP16, 32>(a, s);
        case tc::kPrecTF32: return launch_bwd_t<tc::kPrecTF32, 16>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

int tail_tc_chunk(int precision) { return precision == tc::kPrecTF32 ? 16 : 32; }

size_t tail_tc_chunk_bytes(int precision) {
    switch (precision) {
        case tc::kPrecBF16: return Plan<tc::kPrecBF16, 32, false>::kChunk;
        case tc::kPrecFP16: return Plan<tc::kPrecFP16, 32, false>::kChunk;
        case tc::kPrecTF32: return Plan<tc::kPrecTF32, 16, false>::kChunk;
        default: return 0;
    }
}

cudaError_t launch_tail_tc_fwd(const TcArgs& a, cudaStream_t s) {
    if (a.n_points <= 0) return cudaSuccess;
    switch (a.prec) {
        case tc::kPrecBF16: return launch_fwd_t<tc::kPrecBF16, 32>(a, s);
        case tc::kPrecFP16: return launch_fwd_t<tc::kPrecFP16, 32>(a, s);
        case tc::kPrecTF32: return launch_fwd_t<tc::kPrecTF32, 16>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace shs
