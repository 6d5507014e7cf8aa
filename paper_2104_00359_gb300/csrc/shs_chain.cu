// Scene chain above the shading path (Sec. 3.3.1, Sec. 3.5): per array of M
// rows (vertices, normals or sphere centres) a linear deformation model and
// the rigid pose of each of V views,
//   x_rest[m]  = base[m] + basis[m] p        (basis[m]: 3 x D, row-major [M][3][D])
//   x[v][m]    = R(w_v) x_rest[m] + t_v      (t dropped for directions)
// with R(w) = exp([w]x) (Rodrigues' formula), and the adjoint to p and to
// every view's pose (w_v, t_v).  The deformation is computed once per row for
// all views; lane v of the row's warp applies view v.
//
// The basis is the only large operand (M * 3 * D floats), read once per pass:
// one warp per row, lanes striding the D parameters, so each row's 3 D floats
// are read as contiguous 128-byte segments; a warp takes two rows per step and
// issues the next step's loads before reducing the current rows.  The
// adjoint's sums over rows are kept per lane / per warp, combined per block in
// a fixed order, and the blocks' partial rows are added in a fixed order by a
// second kernel spread over SMs (one block per 32 parameters and per view),
// which also turns dL/dR into dL/dw.

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "shs.h"
#include "shs_internal.h"

namespace {

constexpr int kChainWarps = 8;                  // 256-thread blocks
constexpr int kChainThreads = 32 * kChainWarps;
constexpr int kChainMaxD = SHS_CHAIN_MAX_PARAMS;
constexpr int kChainMaxBlocks = 152 * 4;
constexpr int kChainExtra = 12;                 // per view: dL/dR (9, row-major) and dL/dt (3)
constexpr int kChainMaxViews = SHS_CHAIN_MAX_VIEWS;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over lanes 0 .. V-1 (the others hold zeros): log2 of the next power of
// two >= V exchange rounds, then lane 0's total is broadcast.
__device__ __forceinline__ float view_sum(float v, int rounds) {
    for (int o = 1, r = 0; r < rounds; o <<= 1, ++r) v += __shfl_xor_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// R(w) = I + A K + B K^2, K = [w]x, A = sin th / th, B = (1 - cos th) / th^2
// written as 2 sin^2(th/2) / th^2 (no cancellation at small th); series below
// th = 1e-3.
__device__ __forceinline__ void rotation(const float* pose, float* R) {
    const float wx = __ldg(pose), wy = __ldg(pose + 1), wz = __ldg(pose + 2);
    const float t2 = wx * wx + wy * wy + wz * wz;
    float A, B;
    if (t2 < 1e-6f) {
        A = 1.f - t2 * (1.f / 6.f);
        B = 0.5f - t2 * (1.f / 24.f);
    } else {
        const float th = sqrtf(t2);
        float s, c, sh, ch;
        sincosf(th, &s, &c);
        sincosf(0.5f * th, &sh, &ch);
        A = s / th;
        const float q = sh / (0.5f * th);
        B = 0.5f * q * q;
    }
    // K^2 = w w^T - t2 I
    R[0] = 1.f + B * (wx * wx - t2);
    R[1] = -A * wz + B * wx * wy;
    R[2] = A * wy + B * wx * wz;
    R[3] = A * wz + B * wy * wx;
    R[4] = 1.f + B * (wy * wy - t2);
    R[5] = -A * wx + B * wy * wz;
    R[6] = -A * wy + B * wz * wx;
    R[7] = A * wx + B * wz * wy;
    R[8] = 1.f + B * (wz * wz - t2);
}

// Rows per warp and step: all of their basis loads are issued before any is
// used, so a warp keeps RW * 3 * PL independent loads in flight.
#ifndef SHS_CHAIN_ROWS
#define SHS_CHAIN_ROWS 2
#endif
#ifdef SHS_CHAIN_MINB
#define SHS_CHAIN_BOUNDS __launch_bounds__(kChainThreads, SHS_CHAIN_MINB)
#else
#define SHS_CHAIN_BOUNDS __launch_bounds__(kChainThreads)
#endif
constexpr int kChainRowsPerStep = SHS_CHAIN_ROWS;

// PL: parameters per lane (D <= 32 PL).  Loads beyond D or M read nothing and
// count as zero.  poses: [V][6]; x: [V][M][3].
template <int PL>
__global__ void SHS_CHAIN_BOUNDS chain_forward_kernel(const float* base, const float* basis, int64_t M,
                                                      int D, const float* p, const float* poses, int V,
                                                      int direction, float* x_rest, float* x) {
    constexpr int RW = kChainRowsPerStep;
    __shared__ float s_p[32 * PL];
    __shared__ float s_rt[kChainMaxViews][12];      // R (9) and t (3) per view
    for (int d = threadIdx.x; d < 32 * PL; d += kChainThreads) s_p[d] = d < D ? __ldg(p + d) : 0.f;
    if (threadIdx.x < V) {
        const float* pose = poses + 6 * threadIdx.x;
        rotation(pose, s_rt[threadIdx.x]);
        for (int c = 0; c < 3; ++c) s_rt[threadIdx.x][9 + c] = direction ? 0.f : __ldg(pose + 3 + c);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // lane v applies view v (V <= 32)
    float R[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) R[i] = lane < V ? s_rt[lane][i] : 0.f;
    const int64_t step = static_cast<int64_t>(gridDim.x) * kChainWarps * RW;
    // the next step's rows are loaded while this step's are reduced
    auto load = [&](float (*bb)[3][PL], int64_t mb) {
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int64_t m = mb + r;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int j = 0; j < PL; ++j) {
                    const int d = lane + 32 * j;
                    bb[r][c][j] = (m < M && d < D) ? __ldcs(basis + (m * 3 + c) * D + d) : 0.f;
                }
            }
        }
    };
    int64_t m0 = (static_cast<int64_t>(blockIdx.x) * kChainWarps + (threadIdx.x >> 5)) * RW;
    float b[RW][3][PL];
    load(b, m0);
    for (; m0 < M; m0 += step) {
        float bn[RW][3][PL];
        load(bn, m0 + step);
        float acc[RW][3];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float t = 0.f;
#pragma unroll
                for (int j = 0; j < PL; ++j) t = fmaf(b[r][c][j], s_p[lane + 32 * j], t);
                acc[r][c] = warp_sum(t);
            }
        }
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int64_t m = m0 + r;
            if (m >= M) continue;
            const float a0 = acc[r][0] + __ldg(base + 3 * m), a1 = acc[r][1] + __ldg(base + 3 * m + 1),
                        a2 = acc[r][2] + __ldg(base + 3 * m + 2);
            if (x_rest && lane == 0) {
                x_rest[3 * m] = a0;
                x_rest[3 * m + 1] = a1;
                x_rest[3 * m + 2] = a2;
            }
            if (lane < V) {
                float* xo = x + (static_cast<int64_t>(lane) * M + m) * 3;
                xo[0] = fmaf(R[0], a0, fmaf(R[1], a1, fmaf(R[2], a2, R[9])));
                xo[1] = fmaf(R[3], a0, fmaf(R[4], a1, fmaf(R[5], a2, R[10])));
                xo[2] = fmaf(R[6], a0, fmaf(R[7], a1, fmaf(R[8], a2, R[11])));
            }
        }
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int j = 0; j < PL; ++j) b[r][c][j] = bn[r][c][j];
    }
}

// Partial sums of one block: [0, D) dL/dp, then per view dL/dR (9), dL/dt (3).
// d_x: [V][M][3].  Lane v takes view v's gradient of the row: it adds
// R_v^T g_v to the rest-frame gradient (summed over the warp's lanes) and
// accumulates view v's dL/dR and dL/dt.
template <int PL>
__global__ void SHS_CHAIN_BOUNDS chain_backward_kernel(const float* base, const float* basis, int64_t M,
                                                       int D, const float* p, const float* poses, int V,
                                                       int direction, const float* g, float* partials) {
    constexpr int RW = kChainRowsPerStep;
    __shared__ float s_p[32 * PL];
    __shared__ float s_dp[kChainWarps][32 * PL];
    __shared__ float s_ex[kChainWarps][kChainMaxViews][kChainExtra];
    __shared__ float s_r[kChainMaxViews][9];
    for (int d = threadIdx.x; d < 32 * PL; d += kChainThreads) s_p[d] = d < D ? __ldg(p + d) : 0.f;
    if (threadIdx.x < V) rotation(poses + 6 * threadIdx.x, s_r[threadIdx.x]);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool view = lane < V;
    int vrounds = 0;
    while ((1 << vrounds) < V) ++vrounds;
    float R[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = view ? s_r[lane][i] : 0.f;
    float dp[PL];
#pragma unroll
    for (int j = 0; j < PL; ++j) dp[j] = 0.f;
    float ex[kChainExtra];
#pragma unroll
    for (int i = 0; i < kChainExtra; ++i) ex[i] = 0.f;
    const int64_t step = static_cast<int64_t>(gridDim.x) * kChainWarps * RW;
    // the next step's rows are loaded while this step's are reduced
    auto load = [&](float (*bb)[3][PL], float (*gb)[3], int64_t mb) {
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int64_t m = mb + r;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gb[r][c] = (m < M && view) ? __ldg(g + (static_cast<int64_t>(lane) * M + m) * 3 + c) : 0.f;
#pragma unroll
                for (int j = 0; j < PL; ++j) {
                    const int d = lane + 32 * j;
                    bb[r][c][j] = (m < M && d < D) ? __ldcs(basis + (m * 3 + c) * D + d) : 0.f;
                }
            }
        }
    };
    int64_t m0 = (static_cast<int64_t>(blockIdx.x) * kChainWarps + warp) * RW;
    float b[RW][3][PL], gg[RW][3];
    load(b, gg, m0);
    for (; m0 < M; m0 += step) {
        float bn[RW][3][PL], gn[RW][3];
        load(bn, gn, m0 + step);
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            // sum over views of R_v^T g_v: the gradient in the rest frame
            const float r0 = view_sum(fmaf(R[0], gg[r][0], fmaf(R[3], gg[r][1], R[6] * gg[r][2])), vrounds);
            const float r1 = view_sum(fmaf(R[1], gg[r][0], fmaf(R[4], gg[r][1], R[7] * gg[r][2])), vrounds);
            const float r2 = view_sum(fmaf(R[2], gg[r][0], fmaf(R[5], gg[r][1], R[8] * gg[r][2])), vrounds);
            float xr[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float t = 0.f;
#pragma unroll
                for (int j = 0; j < PL; ++j) t = fmaf(b[r][c][j], s_p[lane + 32 * j], t);
                xr[c] = warp_sum(t);
            }
#pragma unroll
            for (int j = 0; j < PL; ++j) dp[j] = fmaf(b[r][0][j], r0, fmaf(b[r][1][j], r1, fmaf(b[r][2][j], r2, dp[j])));
            const int64_t m = m0 + r;
            if (m < M) {
#pragma unroll
                for (int c = 0; c < 3; ++c) xr[c] += __ldg(base + 3 * m + c);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) ex[3 * a + c] = fmaf(gg[r][a], xr[c], ex[3 * a + c]);
                    if (!direction) ex[9 + a] += gg[r][a];
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RW; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gg[r][c] = gn[r][c];
#pragma unroll
                for (int j = 0; j < PL; ++j) b[r][c][j] = bn[r][c][j];
            }
    }
#pragma unroll
    for (int j = 0; j < PL; ++j) s_dp[warp][lane + 32 * j] = dp[j];
    if (view) {
#pragma unroll
        for (int i = 0; i < kChainExtra; ++i) s_ex[warp][lane][i] = ex[i];
    }
    __syncthreads();
    const int E = D + kChainExtra * V;
    for (int i = threadIdx.x; i < E; i += kChainThreads) {
        float t = 0.f;
        if (i < D) {
            for (int w = 0; w < kChainWarps; ++w) t += s_dp[w][i];
        } else {
            const int v = (i - D) / kChainExtra, k = (i - D) % kChainExtra;
            for (int w = 0; w < kChainWarps; ++w) t += s_ex[w][v][k];
        }
        partials[static_cast<int64_t>(blockIdx.x) * E + i] = t;
    }
}

// Fixed-order sum of the blocks' partial rows, spread over SMs (one SM
// alone keeps too few loads in flight): block k < ceil(D / 32) sums entries
// 32 k .. 32 k + 31 of dL/dp, block ceil(D / 32) + v the 12 entries of view v
// and then maps its dL/dR to dL/dw_v.  In a block, lane l takes one entry
// and warp w the rows b = w mod 32, in eight independent running sums (their
// loads in flight together); warp 0 adds the warps' sums in order.  Thread a
// < 3 of a view block maps dL/dR to dL/dw_v,a:
// dR/dw_a = A K_a + B (K_a K + K K_a) + (A'/th) w_a K + (B'/th) w_a K^2.
constexpr int kChainReduceThreads = 1024;
__global__ void __launch_bounds__(kChainReduceThreads) chain_reduce_kernel(const float* partials, int nblk, int D,
                                                                           int V, const float* poses, float* d_p,
                                                                           float* d_poses) {
    constexpr int NW = kChainReduceThreads / 32;
    __shared__ float s_ex[kChainExtra];
    __shared__ float s_red[NW][33];
    const int E = D + kChainExtra * V;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ndp = (D + 31) / 32;
    const bool dp_block = static_cast<int>(blockIdx.x) < ndp;
    const int vb = blockIdx.x - ndp;                      // view of a view block
    const int i = dp_block ? blockIdx.x * 32 + lane : D + kChainExtra * vb + lane;
    const bool mine = dp_block ? i < D : lane < kChainExtra;
    float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (mine) {
        for (int b = warp; b < nblk; b += 8 * NW) {
            // unconditional (clamped) loads: all eight are issued before any add
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int bu = b + u * NW < nblk ? b + u * NW : nblk - 1;
                v[u] = partials[static_cast<int64_t>(bu) * E + i];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) t[u] += b + u * NW < nblk ? v[u] : 0.f;
        }
    }
    s_red[warp][lane] = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
    __syncthreads();
    if (warp == 0 && mine) {
        float u = 0.f;
#pragma unroll 8
        for (int w = 0; w < NW; ++w) u += s_red[w][lane];
        if (dp_block) d_p[i] = u;
        else s_ex[lane] = u;
    }
    if (dp_block) return;
    __syncthreads();
    // one thread per rotation-vector component
    const int v = vb, a = threadIdx.x;
    if (a >= 3) return;
    const float* ex = s_ex;
    const float* pose = poses + 6 * v;
    float* d_pose = d_poses + 6 * v;
    // float32 throughout (this part's FP64 latency dominated the reduction):
    // below theta = 0.2 the four factors come from their series (the closed
    // forms cancel there), above from sincos with the half-angle form of
    // 1 - cos.
    const float w[3] = {pose[0], pose[1], pose[2]};
    const float t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    float A, B, dA, dB;
    if (t2 < 0.04f) {
        A = 1.f - t2 * (1.f / 6.f) * (1.f - t2 * (1.f / 20.f) * (1.f - t2 * (1.f / 42.f)));
        B = 0.5f - t2 * (1.f / 24.f) * (1.f - t2 * (1.f / 30.f) * (1.f - t2 * (1.f / 56.f)));
        dA = -1.f / 3.f + t2 * (1.f / 30.f) * (1.f - t2 * (1.f / 28.f));
        dB = -1.f / 12.f + t2 * (1.f / 180.f) * (1.f - t2 * (3.f / 112.f));
    } else {
        const float th = sqrtf(t2);
        float s, c, sh, ch;
        sincosf(th, &s, &c);
        sincosf(0.5f * th, &sh, &ch);
        const float omc = 2.f * sh * sh;                   // 1 - cos theta
        A = s / th;
        B = omc / t2;
        dA = (th * c - s) / (t2 * th);
        dB = (th * s - 2.f * omc) / (t2 * t2);
    }
    // With K = [w]x, K_a = [e_a]x and X = dL/dR (row-major ex[0..8]):
    //   sum K_a o X = X[a2][a1] - X[a1][a2]            (a1, a2 = a + 1, a + 2 mod 3)
    //   K_a K + K K_a = w e_a^T + e_a w^T - 2 w_a I,  so sum (.) o X = (X^T w)_a + (X w)_a - 2 w_a tr X
    //   sum K o X = w . (X[2][1] - X[1][2], X[0][2] - X[2][0], X[1][0] - X[0][1])
    //   sum K^2 o X = w^T X w - t2 tr X
    float X[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) X[e] = ex[e];
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    const float tr = X[0] + X[4] + X[8];
    const float wa = a == 0 ? w[0] : a == 1 ? w[1] : w[2];
    float xw_a = 0.f, xtw_a = 0.f, wxw = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        xw_a = fmaf(ex[3 * a + q], w[q], xw_a);
        xtw_a = fmaf(ex[3 * q + a], w[q], xtw_a);
        float row = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) row = fmaf(X[3 * q + c], w[c], row);
        wxw = fmaf(w[q], row, wxw);
    }
    const float sk = ex[3 * a2 + a1] - ex[3 * a1 + a2];
    const float kx = w[0] * (X[7] - X[5]) + w[1] * (X[2] - X[6]) + w[2] * (X[3] - X[1]);
    const float acc = A * sk + B * (xtw_a + xw_a - 2.f * wa * tr) + dA * wa * kx + dB * wa * (wxw - t2 * tr);
    d_pose[a] = acc;
    d_pose[3 + a] = ex[9 + a];
}

int chain_grid(int64_t M) {
    const int64_t per = static_cast<int64_t>(kChainWarps) * kChainRowsPerStep;
    const int64_t need = (M + per - 1) / per;
    return static_cast<int>(need < kChainMaxBlocks ? (need > 0 ? need : 1) : kChainMaxBlocks);
}

template <template <int> class F, typename... A>
void by_lanes(int D, A&&... args) {
    if (D <= 32) F<1>::go(args...);
    else if (D <= 64) F<2>::go(args...);
    else if (D <= 128) F<4>::go(args...);
    else F<8>::go(args...);
}
// Blocks of `kernel` the device holds at once (one wave): the kernels loop
// over their rows, so a single resident wave avoids paying block start-up per
// four rows.  Falls back to 152 blocks if the occupancy query fails.
template <typename K>
int resident_blocks(K kernel) {
    int dev = 0, sms = 152, per = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kChainThreads, 0) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return 152;
    }
    return sms * per;
}

int clamp_grid(int64_t need, int resident) {
    const int64_t g = need < resident ? need : resident;
    return static_cast<int>(g > 0 ? g : 1);
}

template <int PL> struct Fwd {
    static void go(int64_t need, cudaStream_t s, const float* base, const float* basis, int64_t M, int D,
                   const float* p, const float* poses, int V, int dir, float* xr, float* x) {
        static const int resident = resident_blocks(chain_forward_kernel<PL>);
        chain_forward_kernel<PL><<<clamp_grid(need, resident), kChainThreads, 0, s>>>(base, basis, M, D, p, poses, V,
                                                                                       dir, xr, x);
    }
};
template <int PL> struct Bwd {
    static void go(int64_t need, cudaStream_t s, const float* base, const float* basis, int64_t M, int D,
                   const float* p, const float* poses, int V, int dir, const float* g, float* partials, int* nblk) {
        static const int resident = resident_blocks(chain_backward_kernel<PL>);
        *nblk = clamp_grid(need < kChainMaxBlocks ? need : kChainMaxBlocks, resident);
        chain_backward_kernel<PL><<<*nblk, kChainThreads, 0, s>>>(base, basis, M, D, p, poses, V, dir, g, partials);
    }
};

shs_status check_chain(const float* base, const float* basis, int64_t M, int32_t D, const float* p,
                       const float* poses, int32_t V, int32_t direction) {
    if (M < 0) return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "M < 0"));
    if (D < 1 || D > kChainMaxD)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "D %d not in 1..%d", D, kChainMaxD));
    if (V < 1 || V > kChainMaxViews)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "n_views %d not in 1..%d", V,
                                                         kChainMaxViews));
    if (M > (int64_t(1) << 40) / (3 * static_cast<int64_t>(D) * V))
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "M x 3 x D too large"));
    if (!p || !poses) return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL p or pose"));
    if (M > 0 && (!base || !basis))
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL base or basis"));
    if (direction != 0 && direction != 1)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "direction must be 0 or 1"));
    return SHS_OK;
}

size_t views_workspace_bytes(int64_t n_rows, int32_t n_params, int32_t n_views) {
    if (n_rows < 0 || n_params < 1 || n_params > kChainMaxD || n_views < 1 || n_views > kChainMaxViews) return 0;
    return sizeof(float) * static_cast<size_t>(chain_grid(n_rows)) * (n_params + kChainExtra * n_views);
}

shs_status forward_views(const float* base, const float* basis, int64_t n_rows, int32_t n_params, const float* p,
                         const float* poses, int32_t n_views, int32_t direction, float* x_rest, float* x,
                         void* stream) {
    shs_status st = check_chain(base, basis, n_rows, n_params, p, poses, n_views, direction);
    if (st != SHS_OK) return st;
    if (n_rows == 0) return SHS_OK;
    if (!x) return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL x"));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t per = static_cast<int64_t>(kChainWarps) * kChainRowsPerStep;
    by_lanes<Fwd>(n_params, (n_rows + per - 1) / per, s, base, basis, n_rows, n_params, p, poses, n_views, direction,
                  x_rest, x);
    shs::count_launch();
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, "chain forward"));
}

shs_status backward_views(const float* base, const float* basis, int64_t n_rows, int32_t n_params, const float* p,
                          const float* poses, int32_t n_views, int32_t direction, const float* d_x, float* d_p,
                          float* d_poses, void* workspace, size_t workspace_bytes, void* stream) {
    shs_status st = check_chain(base, basis, n_rows, n_params, p, poses, n_views, direction);
    if (st != SHS_OK) return st;
    if (!d_p || !d_poses || !workspace)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL d_p, d_pose or workspace"));
    if (n_rows > 0 && !d_x) return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL d_x"));
    if (reinterpret_cast<uintptr_t>(workspace) & 15u)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "workspace not 16-byte aligned"));
    const size_t need = views_workspace_bytes(n_rows, n_params, n_views);
    if (workspace_bytes < need)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "workspace of %zu bytes < %zu needed",
                                                         workspace_bytes, need));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* partials = static_cast<float*>(workspace);
    int nblk = 0;
    if (n_rows > 0) {
        const int64_t per = static_cast<int64_t>(kChainWarps) * kChainRowsPerStep;
        by_lanes<Bwd>(n_params, (n_rows + per - 1) / per, s, base, basis, n_rows, n_params, p, poses, n_views,
                      direction, d_x, partials, &nblk);
        shs::count_launch();
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return static_cast<shs_status>(shs::report_cuda(e, "chain backward"));
    }
    chain_reduce_kernel<<<(n_params + 31) / 32 + n_views, kChainReduceThreads, 0, s>>>(partials, nblk, n_params,
                                                                                        n_views, poses, d_p, d_poses);
    shs::count_launch();
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, "chain reduce"));
}

}  // namespace

extern "C" size_t shs_chain_workspace_bytes(int64_t n_rows, int32_t n_params) {
    return views_workspace_bytes(n_rows, n_params, 1);
}

extern "C" size_t shs_chain_views_workspace_bytes(int64_t n_rows, int32_t n_params, int32_t n_views) {
    return views_workspace_bytes(n_rows, n_params, n_views);
}

extern "C" shs_status shs_chain_forward(const float* base, const float* basis, int64_t n_rows, int32_t n_params,
                                        const float* p, const float* pose, int32_t direction, float* x_rest,
                                        float* x, void* stream) {
    return forward_views(base, basis, n_rows, n_params, p, pose, 1, direction, x_rest, x, stream);
}

extern "C" shs_status shs_chain_forward_views(const float* base, const float* basis, int64_t n_rows,
                                              int32_t n_params, const float* p, const float* poses,
                                              int32_t n_views, int32_t direction, float* x_rest, float* x,
                                              void* stream) {
    return forward_views(base, basis, n_rows, n_params, p, poses, n_views, direction, x_rest, x, stream);
}

extern "C" shs_status shs_chain_backward(const float* base, const float* basis, int64_t n_rows, int32_t n_params,
                                         const float* p, const float* pose, int32_t direction, const float* d_x,
                                         float* d_p, float* d_pose, void* workspace, size_t workspace_bytes,
                                         void* stream) {
    return backward_views(base, basis, n_rows, n_params, p, pose, 1, direction, d_x, d_p, d_pose, workspace,
                          workspace_bytes, stream);
}

extern "C" shs_status shs_chain_backward_views(const float* base, const float* basis, int64_t n_rows,
                                               int32_t n_params, const float* p, const float* poses,
                                               int32_t n_views, int32_t direction, const float* d_x, float* d_p,
                                               float* d_poses, void* workspace, size_t workspace_bytes,
                                               void* stream) {
    return backward_views(base, basis, n_rows, n_params, p, poses, n_views, direction, d_x, d_p, d_poses, workspace,
                          workspace_bytes, stream);
}
