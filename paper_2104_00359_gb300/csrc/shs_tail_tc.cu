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
// Projected exponential (variant 1).  V = e0 P[exp(f^)] by the 2n x 4n rule
// (16 Gauss-Legendre nodes x 32 azimuths, 512 directions) is one pass of the
// same form: X = f^ Y^T, U = (exp(X) o w) Y, exp on the CUDA cores in place
// of the square.  The rule is exact to degree 31, so the shading pass (and
// in the adjoint its projections) runs through it too: one table set of 512
// directions, streamed.  The adjoint's last pass is
// df^ = P[exp(f^ Y^T) o (dU Y^T)], with dU = e0 dV.
//
// Roles in a block of 288 threads: warps 0-7 are the compute warps, two
// threads per point (tensor-memory lane): warps w and w + 4 read lanes
// 32 (w % 4) .. + 31 and take the two halves of each chunk's columns and of
// each per-point operand row; both keep the point's full exponent state.  They
// set up the exponent, square and split the GEMM outputs and run the
// direction sums (the first half alone).  Lane 0 of warp 8 issues the MMAs
// and the table copies.  Hand-offs go through mbarriers; every wait is bounded (about
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
constexpr int kCompute = 256;     // compute threads: two per point (one per half of each chunk)
constexpr int kThreads = 288;     // + the MMA / copy warp
constexpr int kMmaWarp = kCompute / 32;
constexpr int kSmemBudget = 227 * 1024;
using SH = shsgen::SH<8>;

// Directions per table chunk: the forward streams wider chunks (its operands
// live in tensor memory), the adjoint narrower ones (two operand rows and the
// chunk operands share shared memory with the ring).
constexpr int kCqFwdBF16 = 64, kCqFwdFP16 = 64, kCqFwdTF32 = 32;
constexpr int kCqBwdBF16 = 32, kCqBwdFP16 = 32, kCqBwdTF32 = 16;


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

// Directions of a variant's rule.
template <int VAR>
constexpr int rule_dirs() {
    return VAR ? kTcQExp : kTcQ;
}

// Direction table: s_dir[q] = (x, y, z, w_q), s_lc[c][q] = L_c(w_q).
template <int Q>
__device__ void load_directions(const TcArgs& a, float4* s_dir, float (*s_lc)[Q]) {
    for (int q = threadIdx.x; q < Q; q += kCompute) {
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
    asm volatile("bar.sync 1, 256;" ::: "memory");
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

// Projected exponential: one pass (k = 1) evaluates and projects exp(f^);
// S = f^, f without its constant term.
__device__ __forceinline__ ExpState proj_setup(float* S) {
    ExpState x;
    x.k = 1;
    x.e0 = expf(S[0] * kInvSqrt4Pi);
    x.scale = 1.f;
    x.nrm2 = 0.f;
    x.ol = OLCoef{1.f, 1.f, 0.f, 0.f};
    S[0] = 0.f;
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
    // With as many stages as chunks the tables stay resident: each chunk is
    // copied once and its stage's barrier completes once (phase 0).
    static constexpr bool kResident = R >= NCH;
    uint64_t* full;
    uint64_t* empty;
    unsigned char* base;
    const unsigned char* src;
    uint32_t issued = 0;

    __device__ static uint32_t full_parity(uint32_t s) { return kResident ? 0u : (s / R) & 1u; }

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
        if (kResident) return true;
        while (issued <= seq)
            if (!load_next(abort, status)) return false;
        return true;
    }
    // After step seq committed the release of chunk seq - 1: refill the stage
    // released a step earlier (chunk seq - 2), if not done yet.
    __device__ bool refill(uint32_t seq, volatile int* abort, int* status) {
        if (kResident || seq < 2 || issued > seq - 2 + R) return true;
        return load_next(abort, status);
    }
    __device__ unsigned char* stage(uint32_t s) const { return base + (s % R) * CHUNK; }
    // Wait (bounded, ignoring aborts) for every copy still in flight.
    __device__ void drain(uint32_t consumed) {
        if (kResident) {
            for (uint32_t s = 0; s < static_cast<uint32_t>(R); ++s) (void)tc::mbar_wait(&full[s], 0u);
            return;
        }
        for (uint32_t s = consumed; s < issued; ++s) (void)tc::mbar_wait(&full[s % R], (s / R) & 1u);
    }
};

// ---------------------------------------------------------------------------
// forward tail
// ---------------------------------------------------------------------------
// The per-point operands live in tensor memory (the MMAs read A from there):
// shared memory holds only the tables, resident for BF16 / FP16 (all chunks)
// and streamed through a ring for TF32.  Tensor-memory columns: the split S
// (kTmS), two fp32 buffers of X = S Y_c^T (kTmX), two split (X o X) operands
// (kTmXs), the accumulator S' (kTmAcc).
template <int PR, int CQ, int Q>
struct PlanF {
    using P = tc::Prec<PR>;
    static constexpr int EB = P::kElem, NP = P::kParts;
    static constexpr int NCH = Q / CQ;
    static constexpr uint32_t kTb = CQ * 64u * EB;       // one part of Y_c or (wY)_c
    static constexpr uint32_t kChunk = 2u * NP * kTb;
    static constexpr uint32_t kOffDir = 0;
    static constexpr uint32_t kOffRing = Q * 28;          // float4 dir, 3 floats of light
    static constexpr int kStatic = 4096;
    static constexpr int R0 = static_cast<int>((kSmemBudget - kStatic - kOffRing) / kChunk);
    static constexpr int R = R0 >= NCH ? NCH : (R0 > 6 ? 6 : R0);
    static_assert(R >= 3, "table ring needs three stages");
    static constexpr uint32_t kBytes = kOffRing + R * kChunk;
    static constexpr uint32_t kColsS = tc::tmem_cols<PR>(64);      // one part of S
    static constexpr uint32_t kColsX = tc::tmem_cols<PR>(CQ);      // one part of an (X o X) chunk
    static constexpr uint32_t kTmS = 0;
    static constexpr uint32_t kTmX = kTmS + NP * kColsS;
    static constexpr uint32_t kTmXs = kTmX + 2 * CQ;
    static constexpr uint32_t kTmAcc = kTmXs + 2 * NP * kColsX;
    static_assert(kTmAcc + 64 <= 512, "tensor memory plan");
    static constexpr uint32_t kIdescX = tc::idesc_of<PR>(128, CQ);
    static constexpr uint32_t kIdescS = tc::idesc_of<PR>(128, 64);
};

template <int PR, int CQ, int VAR>
__global__ void __launch_bounds__(kThreads, 1) tail_fwd_tc_kernel(const __grid_constant__ TcArgs a) {
    constexpr int Q = rule_dirs<VAR>();
    using PL = PlanF<PR, CQ, Q>;
    constexpr int NCH = PL::NCH, R = PL::R, NP = PL::NP;
    constexpr int HQ = CQ / 2;   // each of a point's two threads takes half of a chunk's columns
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[R], empty[R], xr[2], xs[2], g2[2], ar, sp, fin, hb, hb2;
    __shared__ uint32_t tmem_base;
    __shared__ int s_kt;
    __shared__ int s_abort;
    __shared__ float s_bx[128][3];
    const int tid = threadIdx.x, warp = tid >> 5;
    float4* s_dir = reinterpret_cast<float4*>(sm + PL::kOffDir);
    float (*s_lc)[Q] = reinterpret_cast<float (*)[Q]>(s_dir + Q);
    unsigned char* sRing = sm + PL::kOffRing;
    volatile int* abort = &s_abort;

    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
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
        tc::mbar_init(&hb, 128);
        tc::mbar_init(&hb2, 128);
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

    if (warp == kMmaWarp) {
        if ((tid & 31) == 0) {
            // ---------------- MMA / copy issuer
            Ring<R, NCH, PL::kChunk> ring{full, empty, sRing, static_cast<const unsigned char*>(a.chunks)};
            ring.prime();
            uint32_t seq = 0, arc = 0, xn = 0;   // xn: xs waits so far (buffer xn & 1)
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
                int kt = 0;
                for (int pass = 0; ok; ++pass) {
                    ok = tc::mbar_wait_or_abort(&ar, arc & 1u, abort, a.sc.status);
                    ++arc;
                    if (!ok) break;
                    tc::fence_after_sync();
                    if (pass == 0) kt = s_kt & 31;
                    const bool shading = pass == kt;
                    for (int c = 0; ok && c <= NCH; ++c) {
                        if (c < NCH) {
                            ok = ring.ensure(seq, abort, a.sc.status) &&
                                 tc::mbar_wait_or_abort(&full[seq % R], ring.full_parity(seq), abort, a.sc.status);
                            if (!ok) break;
                            tc::gemm_split_ts<PR, 64, PL::kColsS, PL::kTb>(tmem + PL::kTmX + (c & 1) * CQ,
                                                                          tmem + PL::kTmS,
                                                                          tc::smem_u32(ring.stage(seq)), PL::kIdescX,
                                                                          false);
                            tc::commit(&xr[c & 1]);
                        }
                        if (c >= 1) {
                            const int b = (c - 1) & 1;
                            ok = tc::mbar_wait_or_abort(&xs[b], (xn >> 1) & 1u, abort, a.sc.status);
                            ++xn;
                            if (!ok) break;
                            tc::fence_after_sync();
                            if (!shading) {
                                tc::gemm_split_ts<PR, CQ, PL::kColsX, PL::kTb>(
                                    tmem + PL::kTmAcc, tmem + PL::kTmXs + b * NP * PL::kColsX,
                                    tc::smem_u32(ring.stage(seq - 1)) + NP * PL::kTb, PL::kIdescS, c - 1 > 0);
                                tc::commit(&g2[b]);
                            }
                            if (!ring.kResident) tc::commit(&empty[(seq - 1) % R]);
                            if (c == NCH && !shading) tc::commit(&sp);
                        }
                        if (c < NCH) {
                            ok = ring.refill(seq, abort, a.sc.status);
                            ++seq;
                        }
                    }
                    if (shading) break;
                }
            }
            ring.drain(seq);
            tc::commit(&fin);
            (void)tc::mbar_wait(&fin, 0);
        }
    } else {
        // ---------------- compute warps
        load_directions<Q>(a, s_dir, s_lc);
        named_sync_compute();
        const int row = tid & 127, half = tid >> 7;
        const uint32_t lane_tm = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
        const Lobe hl{a.lobe_c1, a.lobe_e[0], a.lobe_e[1], a.lobe_e[2], a.lobe_e[3]};
        uint32_t cn = 0, g2n = 0, spc = 0, arc = 0;   // chunks seen, chunks sent to the projection GEMM
        bool ok = true;
        for (int64_t tile = blockIdx.x, it = 0; ok && tile < ntiles; tile += gridDim.x, ++it) {
            const int64_t p = tile * 128 + row;
            const bool live = p < P;
            const int64_t q = live ? p : 0;
            float S[K];
#pragma unroll
            for (int i = 0; i < K; ++i) S[i] = live ? __ldg(a.f + i * P + q) : 0.f;
            const ExpState ex = VAR ? proj_setup(S) : exp_setup(a.sc, S, S);
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
                // this thread's half of the split S (scaled by 2^-sh) into tensor memory
                sh = row_shift(S);
                {
                    float Sd[32];
                    if (half) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) Sd[i] = ldexpf(S[32 + i], -sh);
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i) Sd[i] = ldexpf(S[i], -sh);
                    }
                    tc::tmem_store_split<PR, 32>(lane_tm + PL::kTmS, PL::kColsS, 32 * half, Sd);
                    tc::tmem_wait_st();
                }
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
                    ok = warp_wait(&xr[b], (cn >> 1) & 1u, abort, a.sc.status);
                    ++cn;
                    if (!ok) break;
                    tc::fence_after_sync();
                    float X[HQ];
                    tc::tmem_ld<HQ>(lane_tm + PL::kTmX + b * CQ + half * HQ, X);
                    if (!shading) {
                        if constexpr (VAR) {
                            const float xs = ldexpf(1.f, sh);   // X holds f^ 2^-sh at the directions
#pragma unroll
                            for (int i = 0; i < HQ; ++i) X[i] = expf(X[i] * xs);
                        } else {
#pragma unroll
                            for (int i = 0; i < HQ; ++i) X[i] *= X[i];
                        }
                        if (c >= 2) {
                            ok = warp_wait(&g2[b], ((g2n - 2) >> 1) & 1u, abort, a.sc.status);
                            if (!ok) break;
                        }
                        tc::tmem_store_split<PR, HQ>(lane_tm + PL::kTmXs + b * NP * PL::kColsX, PL::kColsX,
                                                      half * HQ, X);
                        tc::tmem_wait_st();
                        ++g2n;
                    } else {
                        const int q0 = c * CQ + half * HQ;
#pragma unroll
                        for (int i = 0; i < HQ; ++i) {
                            const float4 d = s_dir[q0 + i];
                            const float t = fmaf(ux, d.x, fmaf(uy, d.y, uz * d.z));
                            const float xw = X[i] * lobe(hl, t) * d.w;
                            B0 = fmaf(xw, s_lc[0][q0 + i], B0);
                            B1 = fmaf(xw, s_lc[1][q0 + i], B1);
                            B2 = fmaf(xw, s_lc[2][q0 + i], B2);
                        }
                    }
                    tc::fence_before_sync();
                    tc::mbar_arrive(&xs[b]);
                }
                if (!ok || shading) break;
                ok = warp_wait(&sp, spc & 1u, abort, a.sc.status);
                ++spc;
                if (!ok) break;
                tc::fence_after_sync();
                // tensor-memory loads are warp-collective: every lane loads, then
                // only points that take part in this squaring keep the result
                const bool take = pass < ex.k;
                const float up = VAR ? a.b2_unscale : ldexpf(a.b2_unscale, 2 * sh);
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    float Sn[32];
                    tc::tmem_ld<32>(lane_tm + PL::kTmAcc + 32 * h2, Sn);
#pragma unroll
                    for (int i = 0; i < 32; ++i) S[32 * h2 + i] = take ? Sn[i] * up : S[32 * h2 + i];
                }
                tc::fence_before_sync();
            }
            if (!ok) break;
            // the two halves' direction sums meet in shared memory
            if (half) {
                if (it > 0) {
                    ok = warp_wait(&hb2, (it - 1) & 1, abort, a.sc.status);
                    if (!ok) break;
                }
                s_bx[row][0] = B0;
                s_bx[row][1] = B1;
                s_bx[row][2] = B2;
                tc::mbar_arrive(&hb);
            } else {
                ok = warp_wait(&hb, it & 1, abort, a.sc.status);
                if (!ok) break;
                B0 += s_bx[row][0];
                B1 += s_bx[row][1];
                B2 += s_bx[row][2];
                tc::mbar_arrive(&hb2);
                if (live) {
                    const float s3 = ex.e0 * ldexpf(1.f, sh);
                    a.radiance[3 * q] = __ldg(a.albedo + 3 * q) * B0 * s3;
                    a.radiance[3 * q + 1] = __ldg(a.albedo + 3 * q + 1) * B1 * s3;
                    a.radiance[3 * q + 2] = __ldg(a.albedo + 3 * q + 2) * B2 * s3;
                    if (a.saved_k) a.saved_k[q] = VAR ? 0 : ex.k;
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
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
// adjoint) give df, stored for the pair pass.  The projected exponential
// (variant 1) is the case kt = 1 with exp in place of the square: pass 0
// projects exp(f^), the adjoint pass forms P[exp(f^ Y^T) o (dU Y^T)], which
// is df^ itself.
// Operands in tensor memory as in the forward: A (S_t) and A2 (dS_{t+1}, or
// in the shading pass the second projected operand X_S H), two fp32 buffers
// each of X = A Y_c^T and G = A2 Y_c^T, two split chunk operands Z, and the
// accumulators (the second, W, shares G's columns where they suffice).
template <int PR, int CQ, int Q>
struct PlanB {
    using P = tc::Prec<PR>;
    static constexpr int EB = P::kElem, NP = P::kParts;
    static constexpr int NCH = Q / CQ;
    static constexpr uint32_t kTb = CQ * 64u * EB;
    static constexpr uint32_t kChunk = 2u * NP * kTb;
    static constexpr uint32_t kOffDir = 0;
    static constexpr uint32_t kOffRing = Q * 28;
    static constexpr int kStatic = 8192;
    static constexpr int R0 = static_cast<int>((kSmemBudget - kStatic - kOffRing) / kChunk);
    static constexpr int R = R0 >= NCH ? NCH : (R0 > 6 ? 6 : R0);
    static_assert(R >= 3, "table ring needs three stages");
    static constexpr uint32_t kBytes = kOffRing + R * kChunk;
    static constexpr uint32_t kColsS = tc::tmem_cols<PR>(64);
    static constexpr uint32_t kColsX = tc::tmem_cols<PR>(CQ);
    static constexpr uint32_t kTmA = 0;
    static constexpr uint32_t kTmA2 = kTmA + NP * kColsS;
    static constexpr uint32_t kTmX = kTmA2 + NP * kColsS;
    static constexpr uint32_t kTmG = kTmX + 2 * CQ;
    static constexpr uint32_t kTmZ = kTmG + 2 * CQ;
    static constexpr uint32_t kTmAcc = kTmZ + 2 * NP * kColsX;
    static constexpr uint32_t kTmW = 2 * CQ >= 64 ? kTmG : kTmAcc + 64;
    static_assert((2 * CQ >= 64 ? kTmAcc + 64 : kTmW + 64) <= 512, "tensor memory plan");
    static_assert(2 * NP * kColsX <= NP * kColsS, "shading operands fit in A2's columns");
    static constexpr uint32_t kIdescX = tc::idesc_of<PR>(128, CQ);
    static constexpr uint32_t kIdescS = tc::idesc_of<PR>(128, 64);
};

template <int PR, int CQ, int VAR>
__global__ void __launch_bounds__(kThreads, 1) tail_bwd_tc_kernel(const __grid_constant__ TcArgs a) {
    constexpr int Q = rule_dirs<VAR>();
    using PL = PlanB<PR, CQ, Q>;
    constexpr int NCH = PL::NCH, R = PL::R, NP = PL::NP;
    constexpr int HQ = CQ / 2;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t full[R], empty[R], xr[2], xs[2], g2[2], ar, sp, fin, hb, hb2;
    __shared__ uint32_t tmem_base;
    __shared__ int s_kt;
    __shared__ int s_abort;
    __shared__ float s_dl[4][3 * K + 1];
    __shared__ float s_lsum[3];
    __shared__ float s_bx[128][7];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float4* s_dir = reinterpret_cast<float4*>(sm + PL::kOffDir);
    float (*s_lc)[Q] = reinterpret_cast<float (*)[Q]>(s_dir + Q);
    unsigned char* sRing = sm + PL::kOffRing;
    volatile int* abort = &s_abort;

    if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
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
        tc::mbar_init(&hb, 128);
        tc::mbar_init(&hb2, 128);
        s_kt = 0;
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = tid; e < 4 * (3 * K + 1); e += kThreads) (&s_dl[0][0])[e] = 0.f;   // per lane group
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

    if (warp == kMmaWarp) {
        if (lane == 0) {
            // ---------------- MMA / copy issuer
            Ring<R, NCH, PL::kChunk> ring{full, empty, sRing, static_cast<const unsigned char*>(a.chunks)};
            ring.prime();
            uint32_t seq = 0, arc = 0, xn = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
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
                                 tc::mbar_wait_or_abort(&full[seq % R], ring.full_parity(seq), abort, a.sc.status);
                            if (!ok) break;
                            const uint32_t st = tc::smem_u32(ring.stage(seq));
                            tc::gemm_split_ts<PR, 64, PL::kColsS, PL::kTb>(tmem + PL::kTmX + (c & 1) * CQ,
                                                                          tmem + PL::kTmA, st, PL::kIdescX, false);
                            if (adj)
                                tc::gemm_split_ts<PR, 64, PL::kColsS, PL::kTb>(tmem + PL::kTmG + (c & 1) * CQ,
                                                                              tmem + PL::kTmA2, st, PL::kIdescX,
                                                                              false);
                            tc::commit(&xr[c & 1]);
                        }
                        if (c >= 1) {
                            const int b = (c - 1) & 1;
                            ok = tc::mbar_wait_or_abort(&xs[b], (xn >> 1) & 1u, abort, a.sc.status);
                            ++xn;
                            if (!ok) break;
                            tc::fence_after_sync();
                            const uint32_t wy = tc::smem_u32(ring.stage(seq - 1)) + NP * PL::kTb;
                            tc::gemm_split_ts<PR, CQ, PL::kColsX, PL::kTb>(
                                tmem + PL::kTmAcc, tmem + PL::kTmZ + b * NP * PL::kColsX, wy, PL::kIdescS, c - 1 > 0);
                            if (shade)
                                tc::gemm_split_ts<PR, CQ, PL::kColsX, PL::kTb>(
                                    tmem + PL::kTmW, tmem + PL::kTmA2 + b * NP * PL::kColsX, wy, PL::kIdescS,
                                    c - 1 > 0);
                            tc::commit(&g2[b]);
                            if (!ring.kResident) tc::commit(&empty[(seq - 1) % R]);
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
        load_directions<Q>(a, s_dir, s_lc);
        named_sync_compute();
        const int row = tid & 127, half = tid >> 7, lg = warp & 3;
        const uint32_t lane_tm = tmem + (static_cast<uint32_t>(lg * 32) << 16);
        const Lobe hl{a.lobe_c1, a.lobe_e[0], a.lobe_e[1], a.lobe_e[2], a.lobe_e[3]};
        // per block: [kMaxK][K + 2][128] -- S_t by coefficient, then each half's row shift
        float* hist = a.hist + static_cast<size_t>(blockIdx.x) * (kMaxK * (K + 2) * 128);
        uint32_t cn = 0, g2n = 0, spc = 0, arc = 0;   // chunks seen, chunks sent to the projection GEMM
        float loss_acc = 0.f;
        bool ok = true;
        for (int64_t tile = blockIdx.x, it = 0; ok && tile < ntiles; tile += gridDim.x, ++it) {
            const int64_t p = tile * 128 + row;
            const bool live = p < P;
            const int64_t q = live ? p : 0;
            float V[K];      // S (forward passes), then dS (adjoint passes)
#pragma unroll
            for (int i = 0; i < K; ++i) V[i] = live ? __ldg(a.f + i * P + q) : 0.f;
            const float e0 = expf(V[0] * kInvSqrt4Pi);
            int k = 1;
            float scale = 1.f;
            OLCoef ol{1.f, 1.f, 0.f, 0.f};
            if constexpr (VAR) {
                V[0] = 0.f;   // S_0 = f^
            } else {
                float nrm2 = 0.f;
#pragma unroll
                for (int i = 1; i < K; ++i) nrm2 = fmaf(V[i], V[i], nrm2);
                k = a.k_in ? (live ? min(max(__ldg(a.k_in + q), 0), kMaxK) : 0) : scaling_k(a.sc, nrm2);
                scale = ldexpf(1.f, -k);
                ol = ol_coef(a.sc, nrm2 * scale * scale);
                V[0] = ol.a * kSqrt4Pi;
#pragma unroll
                for (int i = 1; i < K; ++i) V[i] = ol.b * (V[i] * scale);
            }
            atomicMax(&s_kt, static_cast<int>((it << 5) | k));
            float ux = 0.f, uy = 0.f, uz = 1.f, il = 0.f;
            float dB[3] = {0.f, 0.f, 0.f}, u[3] = {0.f, 0.f, 0.f};
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
                    if (a.target) {
                        dB[c] = __ldg(a.radiance_in + 3 * q + c) - __ldg(a.target + 3 * q + c);
                        if (half == 0) loss_acc = fmaf(0.5f * dB[c], dB[c], loss_acc);
                    } else {
                        dB[c] = __ldg(a.d_radiance + 3 * q + c);
                    }
                    u[c] = __ldg(a.albedo + 3 * q + c) * dB[c];
                }
            }
            // scale of D H (the shading adjoint's projected operand): |L_c(w)| <= 1.1 sum |L_c,i|, |H| <= 1.1
            const int sz = [&] {
                const float zb = 1.25f * (fabsf(u[0]) * s_lsum[0] + fabsf(u[1]) * s_lsum[1] + fabsf(u[2]) * s_lsum[2]);
                return zb > 1e-30f ? min(64, max(-64, ilogbf(zb) - 6)) : 0;
            }();
            // direction sums of the shading adjoint: dB_c / (a_c e0 2^sh), dL/de0, dL/dn (unprojected)
            float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float de0 = 0.f;
            int kt = 0, sh = 0, shg = 0;
            for (int pass = 0; ok && pass <= 2 * kt; ++pass) {
                // operands of this pass (kt is still 0 before pass 0's barrier)
                {
                    float Sd[32];
                    if (pass <= kt) {
                        // forward passes and the shading pass: A = S_pass
                        sh = row_shift(V);
                        if (pass == 0 || pass < kt) {
                            // keep this half of S_t and its row shift for the adjoint
                            float* h = hist + static_cast<size_t>(pass) * (K + 2) * 128;
                            if (half) {
#pragma unroll
                                for (int i = 32; i < 64; ++i) h[i * 128 + row] = V[i];
                            } else {
#pragma unroll
                                for (int i = 0; i < 32; ++i) h[i * 128 + row] = V[i];
                            }
                            h[(K + half) * 128 + row] = __int_as_float(sh);
                        }
                        if (half) {
#pragma unroll
                            for (int i = 0; i < 32; ++i) Sd[i] = ldexpf(V[32 + i], -sh);
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i) Sd[i] = ldexpf(V[i], -sh);
                        }
                        tc::tmem_store_split<PR, 32>(lane_tm + PL::kTmA, PL::kColsS, 32 * half, Sd);
                    } else {
                        const int t = 2 * kt - pass;
                        const float* h = hist + static_cast<size_t>(t) * (K + 2) * 128;
                        sh = __float_as_int(h[(K + half) * 128 + row]);
#pragma unroll
                        for (int i = 0; i < 32; ++i) Sd[i] = ldexpf(h[(32 * half + i) * 128 + row], -sh);
                        tc::tmem_store_split<PR, 32>(lane_tm + PL::kTmA, PL::kColsS, 32 * half, Sd);
                        shg = row_shift(V);
                        if (half) {
#pragma unroll
                            for (int i = 0; i < 32; ++i) Sd[i] = ldexpf(V[32 + i], -shg);
                        } else {
#pragma unroll
                            for (int i = 0; i < 32; ++i) Sd[i] = ldexpf(V[i], -shg);
                        }
                        tc::tmem_store_split<PR, 32>(lane_tm + PL::kTmA2, PL::kColsS, 32 * half, Sd);
                    }
                    tc::tmem_wait_st();
                }
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
                    ok = warp_wait(&xr[b], (cn >> 1) & 1u, abort, a.sc.status);
                    ++cn;
                    if (!ok) break;
                    tc::fence_after_sync();
                    float X[HQ];
                    tc::tmem_ld<HQ>(lane_tm + PL::kTmX + b * CQ + half * HQ, X);
                    float Z2[HQ];
                    if (adj) {
                        float G[HQ];
                        tc::tmem_ld<HQ>(lane_tm + PL::kTmG + b * CQ + half * HQ, G);
                        if constexpr (VAR) {
                            const float xs = ldexpf(1.f, sh);
#pragma unroll
                            for (int i = 0; i < HQ; ++i) X[i] = expf(X[i] * xs) * G[i];
                        } else {
#pragma unroll
                            for (int i = 0; i < HQ; ++i) X[i] = 2.f * X[i] * G[i];
                        }
                    } else if (!shade) {
                        if constexpr (VAR) {
                            const float xs = ldexpf(1.f, sh);
#pragma unroll
                            for (int i = 0; i < HQ; ++i) X[i] = expf(X[i] * xs);
                        } else {
#pragma unroll
                            for (int i = 0; i < HQ; ++i) X[i] *= X[i];
                        }
                    } else {
                        // this half's directions: the sums, Z = D H (scaled 2^-sz), Z2 = X H
                        const int q0 = c * CQ + half * HQ;
#pragma unroll
                        for (int i = 0; i < HQ; ++i) {
                            const float4 d = s_dir[q0 + i];
                            const float l0 = s_lc[0][q0 + i], l1 = s_lc[1][q0 + i], l2 = s_lc[2][q0 + i];
                            const float t = fmaf(ux, d.x, fmaf(uy, d.y, uz * d.z));
                            const float hv = lobe(hl, t), hd = lobe_d(hl, t);
                            const float D = fmaf(u[0], l0, fmaf(u[1], l1, u[2] * l2));
                            const float wx = d.w * X[i];
                            const float wxh = wx * hv;
                            acc[0] = fmaf(wxh, l0, acc[0]);
                            acc[1] = fmaf(wxh, l1, acc[1]);
                            acc[2] = fmaf(wxh, l2, acc[2]);
                            acc[3] = fmaf(wxh, D, acc[3]);
                            const float gd = wx * D * hd;
                            acc[4] = fmaf(gd, d.x, acc[4]);
                            acc[5] = fmaf(gd, d.y, acc[5]);
                            acc[6] = fmaf(gd, d.z, acc[6]);
                            Z2[i] = X[i] * hv;
                            X[i] = ldexpf(D * hv, -sz);
                        }
                    }
                    if (c >= 2) {
                        ok = warp_wait(&g2[b], ((g2n - 2) >> 1) & 1u, abort, a.sc.status);
                        if (!ok) break;
                    }
                    tc::tmem_store_split<PR, HQ>(lane_tm + PL::kTmZ + b * NP * PL::kColsX, PL::kColsX, half * HQ, X);
                    if (shade)
                        tc::tmem_store_split<PR, HQ>(lane_tm + PL::kTmA2 + b * NP * PL::kColsX, PL::kColsX, half * HQ,
                                                      Z2);
                    tc::tmem_wait_st();
                    tc::fence_before_sync();
                    tc::mbar_arrive(&xs[b]);
                    ++g2n;
                }
                if (!ok) break;
                ok = warp_wait(&sp, spc & 1u, abort, a.sc.status);
                ++spc;
                if (!ok) break;
                tc::fence_after_sync();
                // the pass's accumulator (S', dV or dS') replaces V where the point takes part
                const bool take = pass < kt ? pass < k : pass == kt ? true : 2 * kt - pass < k;
                const float up = pass < kt ? ldexpf(a.b2_unscale, VAR ? 0 : 2 * sh)
                                           : pass == kt ? e0 * ldexpf(a.b2_unscale, sz)
                                                        : ldexpf(a.b2_unscale, VAR ? shg : sh + shg);
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    float Sn[32];
                    tc::tmem_ld<32>(lane_tm + PL::kTmAcc + 32 * h2, Sn);
#pragma unroll
                    for (int i = 0; i < 32; ++i) V[32 * h2 + i] = take ? Sn[i] * up : V[32 * h2 + i];
                }
                if (shade) {
                    // W = e0 2^sh P[X H]; d_light += u_c W over the points (this half's coefficients)
                    float Wv[32];
                    tc::tmem_ld<32>(lane_tm + PL::kTmW + 32 * half, Wv);
                    tc::fence_before_sync();
                    const float ws = e0 * ldexpf(a.b2_unscale, sh);
#pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        float dl[32];
                        const float uc = live ? u[c3] * ws : 0.f;
#pragma unroll
                        for (int i = 0; i < 32; ++i) dl[i] = uc * Wv[i];
                        warp_sum_into<32>(dl, &s_dl[lg][c3 * K + 32 * half], lane);
                    }
                    // the halves' direction sums meet in shared memory
                    if (half) {
                        if (it > 0) {
                            ok = warp_wait(&hb2, (it - 1) & 1, abort, a.sc.status);
                            if (!ok) break;
                        }
#pragma unroll
                        for (int j = 0; j < 7; ++j) s_bx[row][j] = acc[j];
                        tc::mbar_arrive(&hb);
                    } else {
                        ok = warp_wait(&hb, it & 1, abort, a.sc.status);
                        if (!ok) break;
#pragma unroll
                        for (int j = 0; j < 7; ++j) acc[j] += s_bx[row][j];
                        tc::mbar_arrive(&hb2);
                        const float s2 = ldexpf(1.f, sh);
                        de0 = acc[3] * s2;
                        if (live) {
                            if (a.d_albedo) {
#pragma unroll
                                for (int c3 = 0; c3 < 3; ++c3) a.d_albedo[3 * q + c3] = dB[c3] * e0 * s2 * acc[c3];
                            }
                            if (a.d_normals) {
                                const float gx = e0 * s2 * acc[4], gy = e0 * s2 * acc[5], gz = e0 * s2 * acc[6];
                                const float ug = ux * gx + uy * gy + uz * gz;
                                a.d_normals[3 * q] = (gx - ux * ug) * il;
                                a.d_normals[3 * q + 1] = (gy - uy * ug) * il;
                                a.d_normals[3 * q + 2] = (gz - uz * ug) * il;
                            }
                        }
                    }
                } else {
                    tc::fence_before_sync();
                }
            }
            if (!ok) break;
            // optimal linear step and scaling: S_0 = a(s) sqrt(4 pi), S_i = b(s) g_i, g = f^ 2^-k;
            // each half writes its 32 coefficients of df.  The projected
            // exponential's adjoint pass left df^ itself in V.
            if (live && VAR) {
                if (half == 0) a.dfp_ws[q] = de0 * e0 * kInvSqrt4Pi * a.sc.neg_2pi_eps * SH::norm(0);
#pragma unroll
                for (int i = 1; i < K; ++i) {
                    if ((i >> 5) != half) continue;
                    a.dfp_ws[i * P + q] = V[i] * a.sc.neg_2pi_eps * SH::norm(i);
                }
            } else if (live) {
                float dBs = 0.f;
#pragma unroll
                for (int i = 1; i < K; ++i) dBs = fmaf(V[i], __ldg(a.f + i * P + q) * scale, dBs);
                const float dA = V[0] * kSqrt4Pi;
                const float cg = fmaf(dA, ol.ca, dBs * ol.cb);
                if (half == 0) a.dfp_ws[q] = de0 * e0 * kInvSqrt4Pi * a.sc.neg_2pi_eps * SH::norm(0);
#pragma unroll
                for (int i = 1; i < K; ++i) {
                    if ((i >> 5) != half) continue;
                    const float gi = __ldg(a.f + i * P + q) * scale;
                    a.dfp_ws[i * P + q] = fmaf(ol.b, V[i], cg * gi) * scale * a.sc.neg_2pi_eps * SH::norm(i);
                }
            }
        }
        if (a.target) {
            const float v = warp_sum(loss_acc);
            if (lane == 0) atomicAdd(&s_dl[lg][3 * K], v);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
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

template <int PR, int CQ, int VAR>
cudaError_t launch_fwd_t(const TcArgs& a, cudaStream_t s) {
    using PL = PlanF<PR, CQ, rule_dirs<VAR>()>;
    auto kern = tail_fwd_tc_kernel<PR, CQ, VAR>;
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

template <int PR, int CQ, int VAR>
cudaError_t launch_bwd_t(const TcArgs& a, cudaStream_t s) {
    using PL = PlanB<PR, CQ, rule_dirs<VAR>()>;
    auto kern = tail_bwd_tc_kernel<PR, CQ, VAR>;
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

// The projected exponential takes BF16 or TF32 operands only: exp(f^) spans
// more than the half-precision exponent range.
cudaError_t launch_tail_tc_bwd(const TcArgs& a, cudaStream_t s) {
    if (a.n_points <= 0) return cudaSuccess;
    if (a.variant == 1) {
        switch (a.prec) {
            case tc::kPrecBF16: return launch_bwd_t<tc::kPrecBF16, kCqBwdBF16, 1>(a, s);
            case tc::kPrecTF32: return launch_bwd_t<tc::kPrecTF32, kCqBwdTF32, 1>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (a.variant != 0) return cudaErrorInvalidValue;
    switch (a.prec) {
        case tc::kPrecBF16: return launch_bwd_t<tc::kPrecBF16, kCqBwdBF16, 0>(a, s);
        case tc::kPrecFP16: return launch_bwd_t<tc::kPrecFP16, kCqBwdFP16, 0>(a, s);
        case tc::kPrecTF32: return launch_bwd_t<tc::kPrecTF32, kCqBwdTF32, 0>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

int tail_tc_chunk(int precision, int adjoint) {
    switch (precision) {
        case tc::kPrecBF16: return adjoint ? kCqBwdBF16 : kCqFwdBF16;
        case tc::kPrecFP16: return adjoint ? kCqBwdFP16 : kCqFwdFP16;
        default: return adjoint ? kCqBwdTF32 : kCqFwdTF32;
    }
}

size_t tail_tc_chunk_bytes(int precision, int adjoint) {
    switch (precision) {
        case tc::kPrecBF16:
            return adjoint ? PlanB<tc::kPrecBF16, kCqBwdBF16, kTcQ>::kChunk : PlanF<tc::kPrecBF16, kCqFwdBF16, kTcQ>::kChunk;
        case tc::kPrecFP16:
            return adjoint ? PlanB<tc::kPrecFP16, kCqBwdFP16, kTcQ>::kChunk : PlanF<tc::kPrecFP16, kCqFwdFP16, kTcQ>::kChunk;
        case tc::kPrecTF32:
            return adjoint ? PlanB<tc::kPrecTF32, kCqBwdTF32, kTcQ>::kChunk : PlanF<tc::kPrecTF32, kCqFwdTF32, kTcQ>::kChunk;
        default: return 0;
    }
}

cudaError_t launch_tail_tc_fwd(const TcArgs& a, cudaStream_t s) {
    if (a.n_points <= 0) return cudaSuccess;
    if (a.variant == 1) {
        switch (a.prec) {
            case tc::kPrecBF16: return launch_fwd_t<tc::kPrecBF16, kCqFwdBF16, 1>(a, s);
            case tc::kPrecTF32: return launch_fwd_t<tc::kPrecTF32, kCqFwdTF32, 1>(a, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (a.variant != 0) return cudaErrorInvalidValue;
    switch (a.prec) {
        case tc::kPrecBF16: return launch_fwd_t<tc::kPrecBF16, kCqFwdBF16, 0>(a, s);
        case tc::kPrecFP16: return launch_fwd_t<tc::kPrecFP16, kCqFwdFP16, 0>(a, s);
        case tc::kPrecTF32: return launch_fwd_t<tc::kPrecTF32, kCqFwdTF32, 0>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace shs
