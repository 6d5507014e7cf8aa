// Lighting from an environment map (Eq. 9): L_c,lm = int L_c(w) y_lm(w) dw for
// an equirectangular radiance map, evaluated as the sum over pixels of the
// pixel value times y_lm at the pixel centre times the pixel's exact solid
// angle.
//
// The real SH factor as y_lm(theta, phi) = N'_lm P_l^|m|(cos theta) T_m(phi)
// with T_0 = 1, T_m = cos(m phi), T_-m = sin(m phi) and N'_lm = N_lm (m = 0),
// sqrt(2) N_lm (m != 0).  So each row r of the map first reduces to its 2n-1
// azimuthal moments F_r,c,m = sum_col L_c(r, col) T_m(phi_col) (3 (2n-1)
// multiply-adds per pixel: the pass streams the map once and is bound by HBM),
// and the row then adds dOmega_r N'_lm P_l^|m|(cos theta_r) F_r,c,m to every
// coefficient.  Row sums are per block; a fixed-order pass adds the blocks'
// partial rows, so the result does not depend on scheduling.

#include <cmath>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "shs.h"
#include "shs_internal.h"
#include "shs_warp.cuh"

namespace {

constexpr int kEnvBlock = 128;
constexpr int kEnvMaxBlocks = 152 * 8;
constexpr int kEnvMaxSide = 65536;
constexpr int kEnvReduceWarps = 32;

struct EnvArgs {
    const float* env;        // [H][W][3]
    int H, W;
    const float2* trig;      // [W] (cos, sin) of the column-centre azimuths
    float domega_scale;      // dOmega_r = domega_scale * sin(theta_r)
    float norm[64];          // N'_lm by linear index
    float* partials;         // [gridDim.x][3K]
    int vec4;                // 16-byte aligned map and width % 4 == 0: rows read as float4
    int sym;                 // ... and width % 16 == 0: the four-fold symmetry path (reads the
                             // azimuth table's first W / 4 columns only)
    int trig_ready;          // host side: `trig` already holds the table (the per-width cache)
};

// P_l^m(x) without the Condon-Shortley phase, s = sqrt(1 - x^2) >= 0:
// P_m^m = (2m-1)!! s^m, P_{m+1}^m = (2m+1) x P_m^m,
// (l - m) P_l^m = (2l-1) x P_{l-1}^m - (l+m-1) P_{l-2}^m.
__device__ float assoc_legendre(int l, int m, float x, float s) {
    float pmm = 1.f;
    for (int k = 1; k <= m; ++k) pmm *= (2.f * k - 1.f) * s;
    if (l == m) return pmm;
    float p1 = (2.f * m + 1.f) * x * pmm;
    if (l == m + 1) return p1;
    float p0 = pmm;
    for (int ll = m + 2; ll <= l; ++ll) {
        const float p2 = ((2.f * ll - 1.f) * x * p1 - (ll + m - 1.f) * p0) / (ll - m);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// One pixel's contribution to the 3 (2n-1) azimuthal moments, given
// (cos phi, sin phi).  cos(m phi), sin(m phi) come from repeated rotation by
// phi (complex multiplication: rounding grows about linearly in m, where the
// three-term Chebyshev recurrence amplifies it near phi = 0 and pi); each
// (cos, sin) pair accumulates with one packed float32x2 FMA per channel.
template <int NB>
__device__ __forceinline__ void add_pixel(float v0, float v1, float v2, float c1, float s1, float* acc,
                                          float2* acc2) {
    acc[0] += v0;
    acc[1] += v1;
    acc[2] += v2;
    if constexpr (NB > 1) {
        const float2 w0 = make_float2(v0, v0), w1 = make_float2(v1, v1), w2 = make_float2(v2, v2);
        float cm = c1, sm = s1;
#pragma unroll
        for (int mm = 1; mm < NB; ++mm) {
            const float2 t = make_float2(cm, sm);
            acc2[3 * (mm - 1)] = __ffma2_rn(w0, t, acc2[3 * (mm - 1)]);
            acc2[3 * (mm - 1) + 1] = __ffma2_rn(w1, t, acc2[3 * (mm - 1) + 1]);
            acc2[3 * (mm - 1) + 2] = __ffma2_rn(w2, t, acc2[3 * (mm - 1) + 2]);
            if (mm + 1 < NB) {
                const float cn = fmaf(cm, c1, -sm * s1), sn = fmaf(sm, c1, cm * s1);
                cm = cn;
                sm = sn;
            }
        }
    }
}

// Four columns at once through the azimuthal symmetries of the pixel
// centres: with phi the angle of column c < W/4, the columns W/2 - 1 - c,
// W/2 + c and W - 1 - c sit at pi - phi, pi + phi and -phi, where
//   cos(m (pi + phi)) = (-1)^m cos(m phi),  sin(m (pi + phi)) = (-1)^m sin(m phi),
//   cos(m (-phi)) = cos(m phi),             sin(m (-phi)) = -sin(m phi),
//   cos(m (pi - phi)) = (-1)^m cos(m phi),  sin(m (pi - phi)) = -(-1)^m sin(m phi).
// So with v1..v4 the values at phi, pi + phi, -phi, pi - phi, the four
// pixels add cos(m phi) (v1 + v3 +- (v2 + v4)) and sin(m phi) (v1 - v3 +-
// (v2 - v4)) to the moments (+ for even m, - for odd): one evaluation of the
// harmonics and one multiply-add per moment for four pixels.  cos(m phi),
// sin(m phi) by the recurrence x_{m+1} = 2 cos(phi) x_m - x_{m-1} (for
// m < 8 its rounding error stays within a few tens of ulps).
template <int NB>
__device__ __forceinline__ void add_quad(const float* v1, const float* v2, const float* v3, const float* v4,
                                         float c1, float s1, float* acc, float2* acc2) {
    float ep[3], em[3], sp[3], sm[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float p = v1[ch] + v3[ch], q = v2[ch] + v4[ch], r = v1[ch] - v3[ch], t = v2[ch] - v4[ch];
        ep[ch] = p + q;
        em[ch] = p - q;
        sp[ch] = r + t;
        sm[ch] = r - t;
        acc[ch] += ep[ch];
    }
    if constexpr (NB > 1) {
        const float two_c = c1 + c1;
        float cp = 1.f, spv = 0.f, cm = c1, smv = s1;
#pragma unroll
        for (int mm = 1; mm < NB; ++mm) {
            const float2 t = make_float2(cm, smv);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float2 w = (mm & 1) ? make_float2(em[ch], sm[ch]) : make_float2(ep[ch], sp[ch]);
                acc2[3 * (mm - 1) + ch] = __ffma2_rn(w, t, acc2[3 * (mm - 1) + ch]);
            }
            if (mm + 1 < NB) {
                const float cn = fmaf(two_c, cm, -cp), sn = fmaf(two_c, smv, -spv);
                cp = cm;
                spv = smv;
                cm = cn;
                smv = sn;
            }
        }
    }
}

#ifndef SHS_ENV_MINB
#define SHS_ENV_MINB 4
#endif
#ifndef SHS_ENV_UNROLL
#define SHS_ENV_UNROLL 4
#endif
constexpr int kEnvUnroll = SHS_ENV_UNROLL;
constexpr int kEnvWarps = kEnvBlock / 32;

// One exchange of the halving sum at lane distance O with CNT values left;
// the recursion keeps every index a compile-time constant (the values stay
// in registers).
template <int CNT, int O>
__device__ __forceinline__ void env_transpose_step(float* v, int lane) {
    if constexpr (O > 0) {
        if constexpr (CNT > 1) {
            constexpr int half = CNT / 2;
            const bool up = lane & O;
#pragma unroll
            for (int i = 0; i < half; ++i) {
                const float send = up ? v[i] : v[i + half];
                const float keep = up ? v[i + half] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
            }
            env_transpose_step<half, O / 2>(v, lane);
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
            env_transpose_step<1, O / 2>(v, lane);
        }
    }
}

// Halving-exchange sum of NV values (NV a power of two <= 32): afterwards v[0]
// on lane l holds the warp total of value (l >> (5 - log2 NV)).  Unlike the
// loop form shared by the shading kernels, every index here is a compile-time
// constant, so the values stay in registers (this kernel has them to spare).
template <int NV>
__device__ __forceinline__ void env_transpose_sum(float* v, int lane) {
    env_transpose_step<NV, 16>(v, lane);
}

// Warp total of each of NV values, written to dst[0..NV) by the lanes that
// hold them (halving exchanges over 32, then over the power-of-two rest).
template <int NV>
__device__ __forceinline__ void warp_totals(const float* vals, float* dst, int lane) {
#pragma unroll
    for (int base = 0; base < NV; base += 32) {
        constexpr int R = NV % 32 == 0 ? 32 : NV % 32;
        constexpr int RP = shs::pow2_at_least(R);
        if (NV - base >= 32) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = vals[base + i];
            env_transpose_sum<32>(v, lane);
            dst[base + lane] = v[0];
        } else {
            float v[RP];
#pragma unroll
            for (int i = 0; i < RP; ++i) v[i] = i < R ? vals[base + i] : 0.f;
            env_transpose_sum<RP>(v, lane);
            constexpr int sh = 5 - shs::log2c(RP);
            const int idx = lane >> sh;
            if ((lane & ((1 << sh) - 1)) == 0 && idx < R) dst[base + idx] = v[0];
        }
    }
}

// One warp per map row: the lanes stream the row (4 pixels per lane and
// step, kEnvUnroll steps of loads in flight), the warp sums the row's
// moments and each lane adds them, weighted by the row's Legendre factors,
// into the coefficients it owns (e = lane + 32 j).  No block-wide barrier
// per row; the block's warps meet once, at the end, to write the block's
// partial row in a fixed order.
template <int NB>
__global__ void __launch_bounds__(kEnvBlock, SHS_ENV_MINB) envmap_rows_kernel(const __grid_constant__ EnvArgs a) {
    constexpr int K = NB * NB, NF = 2 * NB - 1, NV = 3 * NF, NOWN = (3 * K + 31) / 32;
    __shared__ float s_mom[kEnvWarps][NV];
    __shared__ float s_coef[kEnvWarps][3 * K];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float coef[NOWN];
#pragma unroll
    for (int j = 0; j < NOWN; ++j) coef[j] = 0.f;
    const bool vec = a.vec4 != 0;
    const int nwarps = gridDim.x * kEnvWarps;

    for (int r = blockIdx.x * kEnvWarps + warp; r < a.H; r += nwarps) {
        // moments: acc = channel sums (m = 0), acc2[3 (m-1) + ch] = (cos, sin) moments
        float acc[3] = {0.f, 0.f, 0.f};
        float2 acc2[NB > 1 ? 3 * (NB - 1) : 1];
#pragma unroll
        for (int v = 0; v < (NB > 1 ? 3 * (NB - 1) : 1); ++v) acc2[v] = make_float2(0.f, 0.f);
        const float* row = a.env + static_cast<size_t>(r) * a.W * 3;
        if (a.sym) {
            // per lane and step: the 4-column group g of the first quarter of
            // the row and its three mirror groups (3 float4 of the map each)
            const float4* row4 = reinterpret_cast<const float4*>(row);
            const float4* trig4 = reinterpret_cast<const float4*>(a.trig);
            const int q4 = a.W >> 4, w8 = a.W >> 3, w4 = a.W >> 2;
            for (int g = lane; g < q4; g += 32) {
                float A[12], B[12], C[12], D[12];
                const int gg[4] = {g, w8 - 1 - g, w8 + g, w4 - 1 - g};   // phi, pi - phi, pi + phi, -phi
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float4 qa = __ldcs(row4 + 3 * gg[0] + k), qb = __ldcs(row4 + 3 * gg[1] + k),
                                 qc = __ldcs(row4 + 3 * gg[2] + k), qd = __ldcs(row4 + 3 * gg[3] + k);
                    A[4 * k] = qa.x; A[4 * k + 1] = qa.y; A[4 * k + 2] = qa.z; A[4 * k + 3] = qa.w;
                    B[4 * k] = qb.x; B[4 * k + 1] = qb.y; B[4 * k + 2] = qb.z; B[4 * k + 3] = qb.w;
                    C[4 * k] = qc.x; C[4 * k + 1] = qc.y; C[4 * k + 2] = qc.z; C[4 * k + 3] = qc.w;
                    D[4 * k] = qd.x; D[4 * k + 1] = qd.y; D[4 * k + 2] = qd.z; D[4 * k + 3] = qd.w;
                }
                const float4 t0 = __ldg(trig4 + 2 * g), t1 = __ldg(trig4 + 2 * g + 1);
                const float tc[4] = {t0.x, t0.z, t1.x, t1.z}, ts[4] = {t0.y, t0.w, t1.y, t1.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)   // column 4g + j; its mirrors sit at 3 - j in B and D
                    add_quad<NB>(&A[3 * j], &C[3 * j], &D[3 * (3 - j)], &B[3 * (3 - j)], tc[j], ts[j], acc, acc2);
            }
        } else if (vec) {
            // 4 pixels (3 float4 of the map, 2 float4 of the azimuth table) per lane and step
            const float4* row4 = reinterpret_cast<const float4*>(row);
            const float4* trig4 = reinterpret_cast<const float4*>(a.trig);
            const int groups = a.W >> 2;
#pragma unroll kEnvUnroll
            for (int g = lane; g < groups; g += 32) {
                const float4 q0 = __ldcs(row4 + 3 * g), q1 = __ldcs(row4 + 3 * g + 1), q2 = __ldcs(row4 + 3 * g + 2);
                const float4 t0 = __ldg(trig4 + 2 * g), t1 = __ldg(trig4 + 2 * g + 1);
                add_pixel<NB>(q0.x, q0.y, q0.z, t0.x, t0.y, acc, acc2);
                add_pixel<NB>(q0.w, q1.x, q1.y, t0.z, t0.w, acc, acc2);
                add_pixel<NB>(q1.z, q1.w, q2.x, t1.x, t1.y, acc, acc2);
                add_pixel<NB>(q2.y, q2.z, q2.w, t1.z, t1.w, acc, acc2);
            }
        } else {
#pragma unroll 4
            for (int col = lane; col < a.W; col += 32) {
                const float2 t = __ldg(a.trig + col);
                add_pixel<NB>(__ldcs(row + 3 * col), __ldcs(row + 3 * col + 1), __ldcs(row + 3 * col + 2), t.x, t.y,
                              acc, acc2);
            }
        }
        // moment v in the kernel's order: channel ch, T index f -> ch * NF + f
        float mom[NV];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            mom[ch * NF] = acc[ch];
#pragma unroll
            for (int mm = 1; mm < NB; ++mm) {
                mom[ch * NF + 2 * mm - 1] = acc2[3 * (mm - 1) + ch].x;
                mom[ch * NF + 2 * mm] = acc2[3 * (mm - 1) + ch].y;
            }
        }
        warp_totals<NV>(mom, s_mom[warp], lane);
        __syncwarp();
        float st, ct;
        sincospif((r + 0.5f) / a.H, &st, &ct);
        const float w_row = a.domega_scale * st;
#pragma unroll
        for (int j = 0; j < NOWN; ++j) {
            const int e = lane + 32 * j;
            if (e < 3 * K) {
                const int ch = e / K, idx = e % K;
                int l = 0;
                while ((l + 1) * (l + 1) <= idx) ++l;
                const int m = idx - l * l - l, am = m < 0 ? -m : m;
                const int f = m == 0 ? 0 : (m > 0 ? 2 * m - 1 : 2 * am);   // moment index of T_m
                coef[j] = fmaf(w_row * a.norm[idx] * assoc_legendre(l, am, ct, st), s_mom[warp][ch * NF + f], coef[j]);
            }
        }
        __syncwarp();   // s_mom[warp] is rewritten by the warp's next row
    }
#pragma unroll
    for (int j = 0; j < NOWN; ++j) {
        const int e = lane + 32 * j;
        if (e < 3 * K) s_coef[warp][e] = coef[j];
    }
    __syncthreads();
    for (int e = tid; e < 3 * K; e += kEnvBlock) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < kEnvWarps; ++w) t += s_coef[w][e];
        a.partials[static_cast<size_t>(blockIdx.x) * (3 * K) + e] = t;
    }
}

// (cos, sin) of the centre azimuth (c + 1/2) 2 pi / W of columns c < n,
// evaluated in double precision and rounded once; small blocks spread the
// (slow, latency-bound) double-precision work over many SMs.
constexpr int kEnvTrigBlock = 64;
__global__ void __launch_bounds__(kEnvTrigBlock) envmap_trig_kernel(int W, int n, float2* trig) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double s, co;
    sincospi((2.0 * c + 1.0) / W, &s, &co);
    trig[c] = make_float2(static_cast<float>(co), static_cast<float>(s));
}

// light[e] = sum over the nblk partial rows in a fixed order; one block per
// 32 entries, 32 warps striding over the rows, eight rows in flight each.
__global__ void __launch_bounds__(32 * kEnvReduceWarps) envmap_reduce_kernel(const float* partials, int nblk, int E,
                                                                         float* light) {
    __shared__ float s[kEnvReduceWarps][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    float t8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (e < E) {
        for (int b = warp; b < nblk; b += 8 * kEnvReduceWarps) {
            // unconditional (clamped) loads: all eight are issued before any add
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int bu = b + u * kEnvReduceWarps < nblk ? b + u * kEnvReduceWarps : nblk - 1;
                v[u] = partials[static_cast<size_t>(bu) * E + e];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) t8[u] += b + u * kEnvReduceWarps < nblk ? v[u] : 0.f;
        }
    }
    s[warp][lane] = ((t8[0] + t8[1]) + (t8[2] + t8[3])) + ((t8[4] + t8[5]) + (t8[6] + t8[7]));
    __syncthreads();
    if (warp != 0 || e >= E) return;
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kEnvReduceWarps; ++w) t += s[w][lane];
    light[e] = t;
}

// Rows are spread evenly over one wave of warps: R = ceil(H / resident
// warps) rows each, ceil(H / R) warps, at most max_grid blocks (the partial
// rows the workspace holds).
template <int NB>
cudaError_t launch_env(EnvArgs& a, int max_grid, float* light, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0 == cudaSuccess)
        e0 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, envmap_rows_kernel<NB>, kEnvBlock, 0);
    if (e0 != cudaSuccess) return e0;
    const long long cap = static_cast<long long>(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1) * kEnvWarps;
    const long long rows_per_warp = (a.H + cap - 1) / cap;
    const long long warps = (a.H + rows_per_warp - 1) / rows_per_warp;
    long long g = (warps + kEnvWarps - 1) / kEnvWarps;
    const int grid = static_cast<int>(g < max_grid ? g : max_grid);
    if (!a.trig_ready) {
        const int ntrig = a.sym ? a.W >> 2 : a.W;   // the symmetry path reads the first quarter
        envmap_trig_kernel<<<(ntrig + kEnvTrigBlock - 1) / kEnvTrigBlock, kEnvTrigBlock, 0, s>>>(
            a.W, ntrig, const_cast<float2*>(a.trig));
        shs::count_launch();
        e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    envmap_rows_kernel<NB><<<grid, kEnvBlock, 0, s>>>(a);
    shs::count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int E = 3 * NB * NB;
    envmap_reduce_kernel<<<(E + 31) / 32, 32 * kEnvReduceWarps, 0, s>>>(a.partials, grid, E, light);
    shs::count_launch();
    return cudaGetLastError();
}

int env_grid(int height) { return height < kEnvMaxBlocks ? height : kEnvMaxBlocks; }

// Azimuth tables kept per device and map width (they depend on nothing
// else), so repeated projections of same-width maps skip the table launch.
// A table is built once, on the caller's stream, which is then synchronised
// so that calls on any stream may read it; a full cache (kEnvTrigCache
// widths per device) leaves further widths to the workspace.
constexpr int kEnvTrigCache = 8;
struct TrigEntry {
    int width = 0;
    float2* table = nullptr;
};
TrigEntry g_trig[64][kEnvTrigCache];
std::mutex g_trig_mutex;

const float2* cached_trig(int width, cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_trig_mutex);
    for (auto& t : g_trig[dev])
        if (t.table && t.width == width) return t.table;
    for (auto& t : g_trig[dev]) {
        if (t.table) continue;
        float2* tab = nullptr;
        if (cudaMalloc(&tab, sizeof(float2) * static_cast<size_t>(width)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        envmap_trig_kernel<<<(width + kEnvTrigBlock - 1) / kEnvTrigBlock, kEnvTrigBlock, 0, s>>>(width, width, tab);
        shs::count_launch();
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(tab);
            return nullptr;
        }
        t.width = width;
        t.table = tab;
        return tab;
    }
    return nullptr;
}

double factorial_ratio(int l, int m) {   // (l - m)! / (l + m)!
    double r = 1.0;
    for (int k = l - m + 1; k <= l + m; ++k) r /= k;
    return r;
}

}  // namespace

// Workspace: the azimuth table [W] float2 (16-byte aligned length), then the
// blocks' partial rows [grid][3K].
size_t trig_bytes(int width) { return (sizeof(float2) * static_cast<size_t>(width) + 255) / 256 * 256; }

extern "C" size_t shs_envmap_workspace_bytes(int32_t height, int32_t width, int32_t n_bands) {
    if (height < 1 || width < 1 || n_bands < 1 || n_bands > 8 || height > kEnvMaxSide || width > kEnvMaxSide)
        return 0;
    return trig_bytes(width) + sizeof(float) * static_cast<size_t>(env_grid(height)) * 3 * n_bands * n_bands;
}

extern "C" shs_status shs_project_envmap(const float* env, int32_t height, int32_t width, int32_t n_bands,
                                         float* light, void* workspace, size_t workspace_bytes, void* stream) {
    if (!env || !light || !workspace)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL env, light or workspace"));
    if (n_bands < 1 || n_bands > 8)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "n_bands %d not in 1..8", n_bands));
    if (height < 1 || width < 1 || height > kEnvMaxSide || width > kEnvMaxSide)
        return static_cast<shs_status>(
            shs::report_error(SHS_ERR_INVALID_ARG, "map %d x %d outside 1..%d per side", height, width, kEnvMaxSide));
    if (workspace_bytes < shs_envmap_workspace_bytes(height, width, n_bands))
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "workspace of %zu bytes < %zu needed",
                                                         workspace_bytes,
                                                         shs_envmap_workspace_bytes(height, width, n_bands)));
    if (reinterpret_cast<uintptr_t>(workspace) & 15u)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "workspace not 16-byte aligned"));
    EnvArgs a{};
    a.env = env;
    a.H = height;
    a.W = width;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float2* cached = cached_trig(width, s);
    a.trig = cached ? cached : static_cast<const float2*>(workspace);
    a.trig_ready = cached ? 1 : 0;
    // cos theta_r - cos theta_{r+1} = 2 sin(theta_r) sin(pi / 2H)
    a.domega_scale = static_cast<float>(2.0 * std::sin(M_PI / (2.0 * height)) * 2.0 * M_PI / width);
    for (int l = 0; l < n_bands; ++l)
        for (int m = -l; m <= l; ++m) {
            const int am = m < 0 ? -m : m;
            const double N = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial_ratio(l, am));
            a.norm[l * l + l + m] = static_cast<float>(m == 0 ? N : std::sqrt(2.0) * N);
        }
    a.partials = reinterpret_cast<float*>(static_cast<unsigned char*>(workspace) + trig_bytes(width));
    // rows of 4k pixels are 48k bytes, so an aligned map keeps every row aligned
    a.vec4 = (width % 4 == 0 && (reinterpret_cast<uintptr_t>(env) & 15u) == 0) ? 1 : 0;
    a.sym = (a.vec4 && width % 16 == 0) ? 1 : 0;
    const int grid = env_grid(height);
    cudaError_t e = cudaSuccess;
    switch (n_bands) {
        case 1: e = launch_env<1>(a, grid, light, s); break;
        case 2: e = launch_env<2>(a, grid, light, s); break;
        case 3: e = launch_env<3>(a, grid, light, s); break;
        case 4: e = launch_env<4>(a, grid, light, s); break;
        case 5: e = launch_env<5>(a, grid, light, s); break;
        case 6: e = launch_env<6>(a, grid, light, s); break;
        case 7: e = launch_env<7>(a, grid, light, s); break;
        default: e = launch_env<8>(a, grid, light, s); break;
    }
    return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, "project envmap"));
}
