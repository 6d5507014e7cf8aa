// Forward and adjoint shading kernels for one band count, compiled once per
// n_bands with -DSHS_NB=n.
//
// Forward (Sec. 3.2-3.3, Eq. 8-13), one thread per shading point:
//   f(x)  = sum_j rotate( ZH of log V'_j , (c_j - x)/|c_j - x| )     pair loop
//   V(x)  = exp*(f)   (DC isolation, 2^-k scaling, optimal linear step,
//                      k squarings with the triple product)
//   H(x)  = rotate( ZH of max(z, 0), n(x) )
//   B_c   = a_c * L_c . (V * H)
// Adjoint: the same steps in reverse, recomputing each sphere's terms instead
// of storing them; scene gradients are reduced warp -> block -> scene scratch.
//
// Per-sphere log-visibility (Sec. 3.3.2, Eq. 13): with s = sin(alpha) =
// min(r / D, 1) and c = cos(alpha), the ZH of -eps * 1[w_z >= c] has
// coefficients -2 pi eps N_l0 int_c^1 P_l(t) dt, and rotating to direction s_hat
// gives F_lm = -2 pi eps (int_c^1 P_l) y_lm(s_hat).  The integral is
//   int_c^1 P_0 = 1 - c,   int_c^1 P_l = (1 - c^2) P_l'(c) / (l (l + 1))  (l >= 1),
// both from Legendre's equation; d/dc int_c^1 P_l = -P_l(c).

#include <type_traits>
#include <cstdint>
#include <cuda_runtime.h>

#include "generated/shs_sh_gen.cuh"
#include "shs_internal.h"
#include "shs_exp.cuh"
#include "shs_warp.cuh"
#include "shs_tc.cuh"

#ifndef SHS_NB
#error "compile with -DSHS_NB=<n_bands>"
#endif

namespace shs {
namespace {

constexpr int NB = SHS_NB;
constexpr int K = NB * NB;
constexpr int KPAD = (K + 3) / 4 * 4;
constexpr int NWARP = kBlock / 32;
using SH = shsgen::SH<NB>;


__host__ __device__ constexpr int band_of(int i) {
    int l = 0;
    while ((l + 1) * (l + 1) <= i) ++l;
    return l;
}

__device__ __forceinline__ float fast_sqrt(float x) {   // sqrt(x) = x / sqrt(x), x >= 0
    return x * rsqrtf(fmaxf(x, 1e-30f));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One mbarrier per block tracks the bulk copies that stage a scene (sphere
// array + lighting) into shared memory.  Initialise it once per block.
__device__ void mbar_init(uint64_t* bar) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// Stage a scene with bulk asynchronous copies completing on `bar` (phase
// `parity`, alternating between stagings).  Every thread waits with a bound of
// about one second; the result is block-uniform: false means the copy did not
// complete, the status word is set and the block must not use the data.  The
// caller must have synchronised the block if shared memory held a previous
// scene that threads may still read.
__device__ bool stage_copy(const SceneView& sc, float4* s_sph, float* s_light, uint64_t* bar,
                           uint32_t parity) {
    const uint32_t sph_bytes = static_cast<uint32_t>(sc.n_spheres) * 16u;
    const uint32_t light_bytes = 3u * KPAD * 4u;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     ::"r"(smem_addr(bar)), "r"(sph_bytes + light_bytes) : "memory");
        if (sph_bytes)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                ::"r"(smem_addr(s_sph)), "l"(sc.spheres), "r"(sph_bytes), "r"(smem_addr(bar))
                : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(smem_addr(s_light)), "l"(sc.light), "r"(light_bytes), "r"(smem_addr(bar))
            : "memory");
    }
    bool done = false;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26) && !done; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.b32 %0, 1, 0, p;\n}\n"
            : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
        done = ok != 0;
        if (!done && global_ns() - t0 > 1000000000ull) break;
    }
    const bool any_failed = __syncthreads_or(!done);
    if (any_failed && threadIdx.x == 0) atomicExch(sc.status, kDevTimeout);
    return !any_failed;
}

__device__ bool stage_scene(const SceneView& sc, float4* s_sph, float* s_light, uint64_t* bar) {
    mbar_init(bar);
    return stage_copy(sc, s_sph, s_light, bar, 0u);
}

// Legendre P_l(c) and P_l'(c) for l < NB (Bonnet recurrence and
// P'_{l+1} = P'_{l-1} + (2l+1) P_l).
__device__ __forceinline__ void legendre(float c, float* P, float* dP) {
    P[0] = 1.f;
    dP[0] = 0.f;
    if (NB > 1) {
        P[1] = c;
        dP[1] = 1.f;
    }
#pragma unroll
    for (int l = 1; l + 1 < NB; ++l) {
        P[l + 1] = fmaf((2.f * l + 1.f) / (l + 1.f) * c, P[l], -(float(l) / (l + 1.f)) * P[l - 1]);
        dP[l + 1] = fmaf(2.f * l + 1.f, P[l], dP[l - 1]);
    }
}

// G_l = int_c^1 P_l(t) dt for l < NB; s2 = 1 - c^2 (passed in because it is
// known more accurately than 1 - c*c).
__device__ __forceinline__ void cap_integrals(float c, float s2, const float* dP, float* G) {
    G[0] = 1.f - c;
#pragma unroll
    for (int l = 1; l < NB; ++l) G[l] = s2 * dP[l] * (1.f / float(l * (l + 1)));
}

// Up to 5 bands, G_l and P_l in closed form in s2 = sin^2 alpha and
// c = cos alpha, with c^2 = 1 - s2 substituted (fewer operations than the
// recurrences, and s2 = r^2 / D^2 is the accurately known quantity):
//   G_0 = 1 - c, G_1 = s2/2, G_2 = c s2/2, G_3 = s2 (1/2 - 5 s2/8),
//   G_4 = c s2 (1/2 - 7 s2/8);
//   P_1 = c, P_2 = 1 - 3 s2/2, P_3 = c (1 - 5 s2/2), P_4 = 1 - 5 s2 + 35 s2^2/8.
__device__ __forceinline__ void cap_closed(float c, float s2, float* G, float* P) {   // NB <= 5 only
    G[0] = 1.f - c;
    P[0] = 1.f;
    if constexpr (NB > 1) {
        G[1] = 0.5f * s2;
        P[1] = c;
    }
    if constexpr (NB > 2) {
        G[2] = G[1] * c;
        P[2] = fmaf(-1.5f, s2, 1.f);
    }
    if constexpr (NB > 3) {
        G[3] = s2 * fmaf(-0.625f, s2, 0.5f);
        P[3] = c * fmaf(-2.5f, s2, 1.f);
    }
    if constexpr (NB > 4) {
        G[4] = G[2] * fmaf(-1.75f, s2, 1.f);
        P[4] = fmaf(s2, fmaf(4.375f, s2, -5.f), 1.f);
    }
}

// G_l (and P_l) of one pair.
__device__ __forceinline__ void cap_terms(float c, float s2, float* G, float* P) {
    if constexpr (NB <= 5) {
        cap_closed(c, s2, G, P);
    } else {
        float dP[NB];
        legendre(c, P, dP);
        cap_integrals(c, s2, dP, G);
    }
}

struct PairGeom {
    float dx, dy, dz, invD, invD2, s2, c;
    bool open;
};

// Unit normal of the shading point, used by horizon culling.
struct Normal {
    float x = 0.f, y = 0.f, z = 0.f;
};

__device__ __forceinline__ Normal unit_normal(float nx, float ny, float nz) {
    const float n2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
    const float il = n2 > 0.f ? rsqrtf(n2) : 0.f;
    return Normal{nx * il, ny * il, nz * il};
}

// With CULL (the optional horizon-culling reading), a sphere entirely below
// the tangent plane at x, (c - x) . n_hat < -r, becomes an empty cap: s2 = 0
// and c = 1 make every G_l zero, and a closed cap carries no gradient.
template <bool CULL = false>
__device__ __forceinline__ PairGeom pair_geometry(float px, float py, float pz, float4 sp, Normal u = {}) {
    PairGeom g;
    g.dx = sp.x - px;
    g.dy = sp.y - py;
    g.dz = sp.z - pz;
    const float D2 = fmaf(g.dx, g.dx, fmaf(g.dy, g.dy, g.dz * g.dz));
    g.invD = D2 > 0.f ? rsqrtf(D2) : 0.f;     // D = 0: every term below vanishes
    g.invD2 = g.invD * g.invD;
    const float r2i = sp.w * sp.w * g.invD2;
    g.open = r2i < 1.f;
    g.s2 = fminf(r2i, 1.f);                   // point inside the sphere: hemisphere cap
    g.c = fast_sqrt(1.f - g.s2);
    if constexpr (CULL) {
        if (fmaf(g.dx, u.x, fmaf(g.dy, u.y, g.dz * u.z)) < -sp.w) {
            g.s2 = 0.f;
            g.c = 1.f;
            g.open = false;
        }
    }
    return g;
}

// Up to 5 bands the pair terms are accumulated in the monomial basis: for each
// band l the pair adds G_l(c) x^a y^b z^c (a+b+c = l) at s_hat, and the
// harmonic combination is taken once per point (mono_to_f).  Above 5 bands the
// number of monomials outgrows the registers and the SH basis is accumulated
// directly.
constexpr bool kMono = NB <= 5;
constexpr int NACC = kMono ? SH::NA : K;

// One pair's un-normalised log-visibility terms, added to acc.
template <bool CULL = false>
__device__ __forceinline__ void pair_forward(float px, float py, float pz, float4 sp, float* acc, Normal u = {}) {
    const PairGeom g = pair_geometry<CULL>(px, py, pz, sp, u);
    float P[NB], G[NB];
    cap_terms(g.c, g.s2, G, P);
    const float sx = g.dx * g.invD, sy = g.dy * g.invD, sz = g.dz * g.invD;
    if constexpr (kMono) {
        SH::accumulate(G, sx, sy, sz, acc);
    } else {
        float Y[K];
        SH::ybar(sx, sy, sz, Y);
#pragma unroll
        for (int i = 0; i < K; ++i) acc[i] = fmaf(G[band_of(i)], Y[i], acc[i]);
    }
}

// Two pairs at once in the packed float32x2 instructions of sm_100+, one
// sphere per half of every float2 (same arithmetic as pair_forward).  The
// spheres come interleaved: qa = (x0, x1, y0, y1), qb = (z0, z1, r0, r1).
template <bool CULL = false>
__device__ __forceinline__ void pair_forward2(float2 npx, float2 npy, float2 npz, float4 qa, float4 qb,
                                              float2* acc, Normal u = {}) {
    const float2 one = make_float2(1.f, 1.f), mone = make_float2(-1.f, -1.f);
    const float2 dx = __fadd2_rn(make_float2(qa.x, qa.y), npx);
    const float2 dy = __fadd2_rn(make_float2(qa.z, qa.w), npy);
    const float2 dz = __fadd2_rn(make_float2(qb.x, qb.y), npz);
    const float2 D2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    const float2 invD = make_float2(D2.x > 0.f ? rsqrtf(D2.x) : 0.f, D2.y > 0.f ? rsqrtf(D2.y) : 0.f);
    const float2 r = make_float2(qb.z, qb.w);
    const float2 r2i = __fmul2_rn(__fmul2_rn(r, r), __fmul2_rn(invD, invD));
    float2 s2 = make_float2(fminf(r2i.x, 1.f), fminf(r2i.y, 1.f));
    const float2 om = __ffma2_rn(s2, mone, one);
    float2 c = __fmul2_rn(om, make_float2(rsqrtf(fmaxf(om.x, 1e-30f)), rsqrtf(fmaxf(om.y, 1e-30f))));
    if constexpr (CULL) {   // as in pair_geometry
        const float2 h = __ffma2_rn(dx, make_float2(u.x, u.x),
                                    __ffma2_rn(dy, make_float2(u.y, u.y), __fmul2_rn(dz, make_float2(u.z, u.z))));
        if (h.x < -qb.z) {
            s2.x = 0.f;
            c.x = 1.f;
        }
        if (h.y < -qb.w) {
            s2.y = 0.f;
            c.y = 1.f;
        }
    }
    float2 G[NB];
    G[0] = __ffma2_rn(c, mone, one);
    if constexpr (NB > 1) G[1] = __fmul2_rn(make_float2(0.5f, 0.5f), s2);
    if constexpr (NB > 2) G[2] = __fmul2_rn(G[1], c);
    if constexpr (NB > 3) G[3] = __fmul2_rn(s2, __ffma2_rn(make_float2(-0.625f, -0.625f), s2, make_float2(0.5f, 0.5f)));
    if constexpr (NB > 4) G[4] = __fmul2_rn(G[2], __ffma2_rn(make_float2(-1.75f, -1.75f), s2, one));
    SH::accumulate2(G, __fmul2_rn(dx, invD), __fmul2_rn(dy, invD), __fmul2_rn(dz, invD), acc);
}

// Interleave the staged spheres in place for pair_forward2: entries 2q and
// 2q+1 become (x, x', y, y') and (z, z', r, r'); an odd last sphere stays as
// it is.  The caller synchronises the block before and after.
__device__ __forceinline__ void interleave_sphere_pairs(float4* s_sph, int N) {
    for (int q = threadIdx.x; q < (N >> 1); q += blockDim.x) {
        const float4 a = s_sph[2 * q], b = s_sph[2 * q + 1];
        s_sph[2 * q] = make_float4(a.x, b.x, a.y, b.y);
        s_sph[2 * q + 1] = make_float4(a.z, b.z, a.w, b.w);
    }
}

// Adjoint of one pair given dfp_i = dLoss/df_i * (-2 pi eps) * NORM_i.
// Returns the gradient with respect to the sphere centre (the point gets the
// negative) and the radius.
template <bool CULL = false>
__device__ __forceinline__ void pair_backward(float px, float py, float pz, float4 sp,
                                              const float* dfp, float& gcx, float& gcy,
                                              float& gcz, float& gr, Normal u = {}) {
    const PairGeom g = pair_geometry<CULL>(px, py, pz, sp, u);
    float P[NB], G[NB];
    cap_terms(g.c, g.s2, G, P);
    const float sx = g.dx * g.invD, sy = g.dy * g.invD, sz = g.dz * g.invD;
    float Y[K];
    SH::ybar(sx, sy, sz, Y);
    float dG[NB];
#pragma unroll
    for (int l = 0; l < NB; ++l) dG[l] = 0.f;
    float w[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        dG[band_of(i)] = fmaf(dfp[i], Y[i], dG[band_of(i)]);
        w[i] = dfp[i] * G[band_of(i)];
    }
    float gx, gy, gz;
    SH::ybar_vjp(sx, sy, sz, w, gx, gy, gz);
    float dc = 0.f;
#pragma unroll
    for (int l = 0; l < NB; ++l) dc = fmaf(-dG[l], P[l], dc);
    // c = sqrt(1 - s2): d c / d s2 = -1 / (2 c); clamped caps carry no gradient
    const float ds2 = g.open ? __fdividef(-0.5f * dc, g.c) : 0.f;
    gr = ds2 * 2.f * sp.w * g.invD2;                 // s2 = r^2 / D^2
    const float dD2 = -ds2 * g.s2 * g.invD2;
    const float sg = sx * gx + sy * gy + sz * gz;    // s_hat = d / D: tangential part
    gcx = fmaf(gx - sx * sg, g.invD, 2.f * dD2 * g.dx);
    gcy = fmaf(gy - sy * sg, g.invD, 2.f * dD2 * g.dy);
    gcz = fmaf(gz - sz * sg, g.invD, 2.f * dD2 * g.dz);
}

// Adjoint of one pair through the per-band homogeneous polynomials
// Phi_l(s) = sum_m dfp_lm Hbar_lm(s) (degree l).  The pair's loss term is
// Psi = sum_l G_l(c) Phi_l(s_hat).  Euler's identity s . grad Phi_l = l Phi_l
// makes every needed quantity a dot product with the per-band gradients:
//   a = sum_l G_l grad Phi_l,    b = sum_l (P_l / l) grad Phi_l   (l >= 1)
//   dPsi/dc = -sum_l P_l Phi_l = -(s_hat . b) - Phi_0
//   dPsi/dd = (a - (s_hat . a) s_hat) / D + 2 (dPsi/dD^2) d
// so only the gradient polynomials (degree l-1) are evaluated per pair.
template <bool CULL = false>
__device__ __forceinline__ void pair_backward_grad(float px, float py, float pz, float4 sp,
                                                   const float* gq, float q0, float& gcx,
                                                   float& gcy, float& gcz, float& gr, Normal u = {}) {
    const PairGeom g = pair_geometry<CULL>(px, py, pz, sp, u);
    float P[NB], G[NB];
    cap_terms(g.c, g.s2, G, P);
    const float sx = g.dx * g.invD, sy = g.dy * g.invD, sz = g.dz * g.invD;
    float gx[NB], gy[NB], gz[NB];
    SH::grad_eval(sx, sy, sz, gq, gx, gy, gz);
    float ax = 0.f, ay = 0.f, az = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll
    for (int l = 1; l < NB; ++l) {
        ax = fmaf(G[l], gx[l - 1], ax);
        ay = fmaf(G[l], gy[l - 1], ay);
        az = fmaf(G[l], gz[l - 1], az);
        const float pl = P[l] * (1.f / float(l));
        bx = fmaf(pl, gx[l - 1], bx);
        by = fmaf(pl, gy[l - 1], by);
        bz = fmaf(pl, gz[l - 1], bz);
    }
    const float rad = fmaf(sx, ax, fmaf(sy, ay, sz * az));
    const float dc = -fmaf(sx, bx, fmaf(sy, by, fmaf(sz, bz, q0)));
    // c = sqrt(1 - s2): d c / d s2 = -1 / (2 c); clamped caps carry no gradient
    const float ds2 = g.open ? __fdividef(-0.5f * dc, g.c) : 0.f;
    gr = ds2 * 2.f * sp.w * g.invD2;                      // s2 = r^2 / D^2
    const float coef = -2.f * ds2 * g.s2 * g.invD2;        // 2 dPsi/dD^2
    gcx = fmaf(fmaf(-rad, sx, ax), g.invD, coef * g.dx);
    gcy = fmaf(fmaf(-rad, sy, ay), g.invD, coef * g.dy);
    gcz = fmaf(fmaf(-rad, sz, az), g.invD, coef * g.dz);
}

// Truncated SH triple product o = a * b (Eq. 7) and square o = a * a.
// Up to 6 bands: the unrolled Gaunt contraction of the generated header.
// From 7 bands: a separable quadrature that is exact for these degrees
// (Gauss-Legendre in cos(theta) x uniform azimuths, tables in the generated
// header): per latitude, the operands' azimuthal coefficients
// c_f = sum_i a_i Leg_i (f the harmonic of i), their values at each azimuth,
// the pointwise product accumulated against the harmonics, then projected
// back with the latitude's weight.  Loop code keeps the instruction footprint
// small (the unrolled contraction is ~10^4 instructions per call).  The
// constant (l = 0) parts go separately: with a = a_0 y_0 + a~ and
// y_0 = 1/sqrt(4 pi), a * b = a~ * b~ + y_0 (a_0 b~ + b_0 a~) + y_0 a_0 b_0 e_0
// exactly, so only a~ * b~ runs through the quadrature; the exponential's
// operands are dominated by their constant part, and this keeps the rounding
// of the quadrature sums relative to the small remainder.
__host__ __device__ constexpr int harm_of(int i) {   // 0: 1, 2m-1: cos m phi, 2m: sin m phi
    return (i - band_of(i) * band_of(i) - band_of(i)) == 0
               ? 0
               : ((i - band_of(i) * band_of(i) - band_of(i)) > 0
                      ? 2 * (i - band_of(i) * band_of(i) - band_of(i)) - 1
                      : -2 * (i - band_of(i) * band_of(i) - band_of(i)));
}

#if SHS_NB >= 7
template <bool SQR>
__device__ __noinline__ void quad_product(const float* __restrict__ a, const float* __restrict__ b,
                                          float* __restrict__ o) {
    constexpr int QZ = SH::QZ, QP = SH::QP, QF = SH::QF;
    const float* leg = SH::qleg();
    const float* trig = SH::qtrig();
    const float* qw = SH::qw();
    float A[K], B[SQR ? 1 : K], O[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        A[i] = a[i];
        if constexpr (!SQR) B[i] = b[i];
        O[i] = 0.f;
    }
    const float a0 = A[0], b0 = SQR ? A[0] : B[0];
    A[0] = 0.f;
    if constexpr (!SQR) B[0] = 0.f;
#pragma unroll 1
    for (int za = 0; za < QZ; ++za) {
        float ca[QF], cb[SQR ? 1 : QF], d[QF];
#pragma unroll
        for (int f = 0; f < QF; ++f) {
            ca[f] = 0.f;
            if constexpr (!SQR) cb[f] = 0.f;
            d[f] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const float L = leg[za * K + i];
            ca[harm_of(i)] = fmaf(A[i], L, ca[harm_of(i)]);
            if constexpr (!SQR) cb[harm_of(i)] = fmaf(B[i], L, cb[harm_of(i)]);
        }
#pragma unroll 1
        for (int pb = 0; pb < QP; ++pb) {
            const float* T = trig + pb * QF;
            float va = 0.f, vb = 0.f;
#pragma unroll
            for (int f = 0; f < QF; ++f) {
                va = fmaf(ca[f], T[f], va);
                if constexpr (!SQR) vb = fmaf(cb[f], T[f], vb);
            }
            const float p = SQR ? va * va : va * vb;
#pragma unroll
            for (int f = 0; f < QF; ++f) d[f] = fmaf(p, T[f], d[f]);
        }
        const float w = qw[za];
#pragma unroll
        for (int i = 0; i < K; ++i) O[i] = fmaf(w * leg[za * K + i], d[harm_of(i)], O[i]);
    }
    O[0] = fmaf(kInvSqrt4Pi * a0, b0, O[0]);
#pragma unroll
    for (int i = 1; i < K; ++i) {
        if constexpr (SQR) O[i] = fmaf(2.f * kInvSqrt4Pi * a0, A[i], O[i]);
        else O[i] = fmaf(kInvSqrt4Pi * a0, B[i], fmaf(kInvSqrt4Pi * b0, A[i], O[i]));
    }
#pragma unroll
    for (int i = 0; i < K; ++i) o[i] = O[i];
}
#endif

__device__ __forceinline__ void sh_mul(const float* a, const float* b, float* o) {
#if SHS_NB >= 7
    quad_product<false>(a, b, o);
#else
    SH::mul(a, b, o);
#endif
}

__device__ __forceinline__ void sh_sqr(const float* a, float* o) {
#if SHS_NB >= 7
    quad_product<true>(a, nullptr, o);
#else
    SH::sqr(a, o);
#endif
}

// Projected-exponential variant of the SH exponential: V = e0 P_n[exp(f^)],
// e0 = exp(f_0 y_0), f^ = f without its constant term, by the variant's rule
// (2n Gauss-Legendre nodes in cos(theta) x 4n azimuths, separable as above):
// per latitude the azimuthal coefficients of f^, its value and exp at each
// azimuth, accumulated against the harmonics, projected with the weight.
// U = P_n[exp(f^)] is returned too (the adjoint needs it).
// Inline up to 6 bands (an out-of-line call puts its operand arrays on the
// stack of every kernel that can take this path); out of line above.
#if SHS_NB <= 6
#define SHS_PROJEXP_INLINE __forceinline__
#else
#define SHS_PROJEXP_INLINE __noinline__
#endif
__device__ SHS_PROJEXP_INLINE void proj_exp(const float* __restrict__ f, float* __restrict__ V,
                                            float* __restrict__ U) {
    constexpr int EZ = SH::EZ, EP = SH::EP, QF = 2 * NB - 1;
    const float* leg = SH::eleg();
    const float* trig = SH::etrig();
    const float* qw = SH::ew();
    float F[K], O[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        F[i] = f[i];
        O[i] = 0.f;
    }
#pragma unroll 1
    for (int za = 0; za < EZ; ++za) {
        float c[QF], d[QF];
#pragma unroll
        for (int q = 0; q < QF; ++q) {
            c[q] = 0.f;
            d[q] = 0.f;
        }
#pragma unroll
        for (int i = 1; i < K; ++i) c[harm_of(i)] = fmaf(F[i], leg[za * K + i], c[harm_of(i)]);
#pragma unroll 1
        for (int pb = 0; pb < EP; ++pb) {
            const float* T = trig + pb * QF;
            float v = 0.f;
#pragma unroll
            for (int q = 0; q < QF; ++q) v = fmaf(c[q], T[q], v);
            const float E = expf(v);
#pragma unroll
            for (int q = 0; q < QF; ++q) d[q] = fmaf(E, T[q], d[q]);
        }
        const float w = qw[za];
#pragma unroll
        for (int i = 0; i < K; ++i) O[i] = fmaf(w * leg[za * K + i], d[harm_of(i)], O[i]);
    }
    const float e0 = expf(F[0] * kInvSqrt4Pi);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        U[i] = O[i];
        V[i] = e0 * O[i];
    }
}

// Adjoint of proj_exp: df from dV.  df_0 = y_0 e0 (dV . U); for j >= 1,
// df_j = e0 sum_q w_q exp(f^_q) (sum_i dV_i y_i(q)) y_j(q).
__device__ SHS_PROJEXP_INLINE void proj_exp_adjoint(const float* __restrict__ f, const float* __restrict__ U,
                                                    const float* __restrict__ dV, float* __restrict__ df) {
    constexpr int EZ = SH::EZ, EP = SH::EP, QF = 2 * NB - 1;
    const float* leg = SH::eleg();
    const float* trig = SH::etrig();
    const float* qw = SH::ew();
    float F[K], G[K], O[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        F[i] = f[i];
        G[i] = dV[i];
        O[i] = 0.f;
    }
#pragma unroll 1
    for (int za = 0; za < EZ; ++za) {
        float c[QF], g[QF], d[QF];
#pragma unroll
        for (int q = 0; q < QF; ++q) {
            c[q] = 0.f;
            g[q] = 0.f;
            d[q] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const float L = leg[za * K + i];
            if (i > 0) c[harm_of(i)] = fmaf(F[i], L, c[harm_of(i)]);
            g[harm_of(i)] = fmaf(G[i], L, g[harm_of(i)]);
        }
#pragma unroll 1
        for (int pb = 0; pb < EP; ++pb) {
            const float* T = trig + pb * QF;
            float v = 0.f, dv = 0.f;
#pragma unroll
            for (int q = 0; q < QF; ++q) {
                v = fmaf(c[q], T[q], v);
                dv = fmaf(g[q], T[q], dv);
            }
            const float p = expf(v) * dv;
#pragma unroll
            for (int q = 0; q < QF; ++q) d[q] = fmaf(p, T[q], d[q]);
        }
        const float w = qw[za];
#pragma unroll
        for (int i = 1; i < K; ++i) O[i] = fmaf(w * leg[za * K + i], d[harm_of(i)], O[i]);
    }
    const float e0 = expf(F[0] * kInvSqrt4Pi);
    float de0 = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) de0 = fmaf(G[i], U[i], de0);
    df[0] = de0 * e0 * kInvSqrt4Pi;
#pragma unroll
    for (int i = 1; i < K; ++i) df[i] = e0 * O[i];
}

// Clamped-cosine SH for a (not necessarily unit) normal; also returns the unit
// normal and 1/|n| for the adjoint.
__device__ __forceinline__ void cosine_lobe(float nx, float ny, float nz, float* H, float& ux,
                                            float& uy, float& uz, float& inv_len) {
    const float n2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
    inv_len = n2 > 0.f ? rsqrtf(n2) : 0.f;
    ux = nx * inv_len;
    uy = ny * inv_len;
    uz = nz * inv_len;
    float Y[K];
    SH::ybar(ux, uy, uz, Y);
#pragma unroll
    for (int i = 0; i < K; ++i) H[i] = SH::ahat(band_of(i)) * SH::norm(i) * Y[i];
}

// Scale the raw pair sums to the log-visibility f.
__device__ __forceinline__ void finish_f(const SceneView& sc, const float* acc, float* f) {
    float fr[K];
    if constexpr (kMono) {
        SH::mono_to_f(acc, fr);
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) fr[i] = acc[i];
    }
#pragma unroll
    for (int i = 0; i < K; ++i) f[i] = sc.neg_2pi_eps * SH::norm(i) * fr[i];
}

__device__ __forceinline__ float load_or(const float* p, int64_t i, bool live) {
    return live ? __ldg(p + i) : 0.f;
}

// ---------------------------------------------------------------------------
// forward kernel
// ---------------------------------------------------------------------------

// Forward shading of point p of one request (Eq. 8), scene staged in shared
// memory.  MODE kFwdFull: pair terms, exponential and shading; kFwdPairs:
// only the log-visibility f, stored; kFwdTail: f read from the saved state,
// then the exponential and shading (lighting or albedo changed, geometry not).
constexpr int kFwdFull = 0, kFwdPairs = 1, kFwdTail = 2;

template <int MODE = kFwdFull>
__device__ __forceinline__ void forward_point(const FwdArgs& a, const float4* s_sph, const float* s_light,
                                              int64_t p) {
    float f[K];
    if constexpr (MODE == kFwdTail) {
#pragma unroll
        for (int i = 0; i < K; ++i) f[i] = __ldg(a.saved_f + i * a.n_points + p);
    } else {
    const float px = __ldg(a.points + 3 * p), py = __ldg(a.points + 3 * p + 1),
                pz = __ldg(a.points + 3 * p + 2);

    float acc[NACC];
    const int N = a.sc.n_spheres;
    if constexpr (kMono) {
        // spheres interleaved in pairs (interleave_sphere_pairs)
        float2 acc2[NACC];
#pragma unroll
        for (int i = 0; i < NACC; ++i) acc2[i] = make_float2(0.f, 0.f);
        const float2 npx = make_float2(-px, -px), npy = make_float2(-py, -py), npz = make_float2(-pz, -pz);
        if (a.sc.horizon_cull) {
            const Normal u = unit_normal(__ldg(a.normals + 3 * p), __ldg(a.normals + 3 * p + 1),
                                         __ldg(a.normals + 3 * p + 2));
#pragma unroll 1
            for (int q = 0; q < (N >> 1); ++q)
                pair_forward2<true>(npx, npy, npz, s_sph[2 * q], s_sph[2 * q + 1], acc2, u);
#pragma unroll
            for (int i = 0; i < NACC; ++i) acc[i] = acc2[i].x + acc2[i].y;
            if (N & 1) pair_forward<true>(px, py, pz, s_sph[N - 1], acc, u);
        } else {
#pragma unroll 1
            for (int q = 0; q < (N >> 1); ++q) pair_forward2(npx, npy, npz, s_sph[2 * q], s_sph[2 * q + 1], acc2);
#pragma unroll
            for (int i = 0; i < NACC; ++i) acc[i] = acc2[i].x + acc2[i].y;
            if (N & 1) pair_forward(px, py, pz, s_sph[N - 1], acc);
        }
    } else {
#pragma unroll
        for (int i = 0; i < NACC; ++i) acc[i] = 0.f;
        if (a.sc.horizon_cull) {
            const Normal u = unit_normal(__ldg(a.normals + 3 * p), __ldg(a.normals + 3 * p + 1),
                                         __ldg(a.normals + 3 * p + 2));
#pragma unroll 2
            for (int j = 0; j < N; ++j) pair_forward<true>(px, py, pz, s_sph[j], acc, u);
        } else {
#pragma unroll 2
            for (int j = 0; j < N; ++j) pair_forward(px, py, pz, s_sph[j], acc);
        }
    }

    finish_f(a.sc, acc, f);
    if constexpr (MODE == kFwdPairs) {
#pragma unroll
        for (int i = 0; i < K; ++i) a.saved_f[i * a.n_points + p] = f[i];
        return;
    }
    }
    float V[K];
    int k = 0;
    if (a.sc.exp_mode == 1) {
        float U[K];
        proj_exp(f, V, U);
    } else {
        float nrm2 = 0.f;
#pragma unroll
        for (int i = 1; i < K; ++i) nrm2 = fmaf(f[i], f[i], nrm2);
        k = scaling_k(a.sc, nrm2);
        const float scale = ldexpf(1.f, -k);
        const OLCoef ol = ol_coef(a.sc, nrm2 * scale * scale);
        float S[K];
        S[0] = ol.a * kSqrt4Pi;
#pragma unroll
        for (int i = 1; i < K; ++i) S[i] = ol.b * (f[i] * scale);
        for (int t = 0; t < k; ++t) {
            float T[K];
            sh_sqr(S, T);
#pragma unroll
            for (int i = 0; i < K; ++i) S[i] = T[i];
        }
        const float e0 = expf(f[0] * kInvSqrt4Pi);
#pragma unroll
        for (int i = 0; i < K; ++i) V[i] = e0 * S[i];
    }

    float H[K], ux, uy, uz, il;
    cosine_lobe(__ldg(a.normals + 3 * p), __ldg(a.normals + 3 * p + 1), __ldg(a.normals + 3 * p + 2),
                H, ux, uy, uz, il);
    float W[K];
    sh_mul(V, H, W);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float d = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) d = fmaf(s_light[c * KPAD + i], W[i], d);
        a.radiance[3 * p + c] = __ldg(a.albedo + 3 * p + c) * d;
    }
    if (MODE == kFwdFull && a.saved_f) {
#pragma unroll
        for (int i = 0; i < K; ++i) a.saved_f[i * a.n_points + p] = f[i];
        a.saved_k[p] = k;
    }
}

#ifndef SHS_FWD_MINB
#define SHS_FWD_MINB 4
#endif
#ifndef SHS_BWD_MINB
#define SHS_BWD_MINB 3
#endif
// Minimum resident blocks above 4 bands.  From 7 bands four blocks per SM
// (128 registers): the spills this costs are outweighed by the latency the
// extra warps hide (height field, 8 bands: forward 5.65 -> 5.23 ms, backward
// 18.1 -> 16.0 ms against one block's bound; 3, 5 and 6 blocks measured
// slower).  5 and 6 bands keep the compiler's choice.
#ifndef SHS_FWD_MINB_HI
#define SHS_FWD_MINB_HI (SHS_NB >= 7 ? 4 : 1)
#endif
#ifndef SHS_BWD_MINB_HI
#define SHS_BWD_MINB_HI (SHS_NB >= 7 ? 4 : 1)
#endif

template <int MODE>
__global__ void __launch_bounds__(kBlock, NB <= 4 ? SHS_FWD_MINB : SHS_FWD_MINB_HI) forward_kernel_t(FwdArgs a) {
    __shared__ __align__(16) float4 s_sph[kMaxSpheres];
    __shared__ __align__(16) float s_light[3 * KPAD];
    __shared__ __align__(8) uint64_t s_bar;
    if (!stage_scene(a.sc, s_sph, s_light, &s_bar)) return;
    if constexpr (kMono) {
        interleave_sphere_pairs(s_sph, a.sc.n_spheres);
        __syncthreads();
    }
    const int64_t p = static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x;
    if (p >= a.n_points) return;
    forward_point<MODE>(a, s_sph, s_light, p);
}


// ---------------------------------------------------------------------------
// backward kernel
// ---------------------------------------------------------------------------

// Sum four values over the warp; lane l returns the total of value (l >> 3).
__device__ __forceinline__ float warp_sum4(float v0, float v1, float v2, float v3, int lane) {
    const bool h16 = lane & 16;
    float ka = h16 ? v2 : v0, kb = h16 ? v3 : v1;
    ka += __shfl_xor_sync(0xffffffffu, h16 ? v0 : v2, 16);
    kb += __shfl_xor_sync(0xffffffffu, h16 ? v1 : v3, 16);
    const bool h8 = lane & 8;
    float k = h8 ? kb : ka;
    k += __shfl_xor_sync(0xffffffffu, h8 ? ka : kb, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}

// Adjoint of one 128-point tile of one request: per-point outputs are written,
// the scene-level sums are added to the block's shared accumulators
// (s_dl: d_light and loss per warp, s_acc: per warp and sphere).
// CULLM: horizon culling off (0), on (1), or read from the scene per call (2);
// EXPM: the exponential's form: the Gaussian optimal linear step (0), the
// projected exponential (1), the tabulated optimal linear step (3), or the
// scene's exp_mode read per call (2).
template <bool PAIRS = true, int CULLM = 2, int EXPM = 2>
__device__ __forceinline__ void backward_tile(const BwdArgs& a, const float4* s_sph, const float* s_light,
                                              float* s_acc, float (*s_dl)[3 * K + 1], int64_t tile,
                                              int lane, int warp) {
    const int N = a.sc.n_spheres;
    const int64_t P = a.n_points;
    const int64_t p = tile * kBlock + threadIdx.x;
    const bool live = p < P;
    const int64_t q = live ? p : 0;
    const float px = load_or(a.points, 3 * q, live), py = load_or(a.points, 3 * q + 1, live),
                pz = load_or(a.points, 3 * q + 2, live);

    // ---- log-visibility f: saved by the forward pass or recomputed
    float f[K];
    int k;
    if (a.saved_f) {
#pragma unroll
        for (int i = 0; i < K; ++i) f[i] = load_or(a.saved_f, i * P + q, live);
        k = live ? min(max(a.saved_k[q], 0), kMaxK) : 0;   // a foreign buffer cannot overrun hist
    } else {
        float acc[NACC];
#pragma unroll
        for (int i = 0; i < NACC; ++i) acc[i] = 0.f;
        if (CULLM == 1 || (CULLM == 2 && a.sc.horizon_cull)) {
            const Normal u = unit_normal(load_or(a.normals, 3 * q, live), load_or(a.normals, 3 * q + 1, live),
                                         load_or(a.normals, 3 * q + 2, live));
#pragma unroll 2
            for (int j = 0; j < N; ++j) pair_forward<true>(px, py, pz, s_sph[j], acc, u);
        } else {
#pragma unroll 2
            for (int j = 0; j < N; ++j) pair_forward(px, py, pz, s_sph[j], acc);
        }
        finish_f(a.sc, acc, f);
        k = -1;
    }
    float nrm2 = 0.f;
#pragma unroll
    for (int i = 1; i < K; ++i) nrm2 = fmaf(f[i], f[i], nrm2);
    if (k < 0) k = scaling_k(a.sc, nrm2);

    // ---- recompute the exponential, keeping the operand of every squaring
    // (or, for the projected-exponential variant, U = P_n[exp(f^)])
    const bool projexp = EXPM == 2 ? a.sc.exp_mode == 1 : EXPM == 1;
    float scale = 1.f, e0 = 1.f;
    OLCoef ol{1.f, 1.f, 0.f, 0.f};
    float g[K], S[K], V[K], U[K];
    float hist[kMaxK][K];
    if (projexp) {
        proj_exp(f, V, U);
    } else {
        scale = ldexpf(1.f, -k);
        ol = ol_coef<EXPM == 0 ? 0 : EXPM == 3 ? 1 : 2>(a.sc, nrm2 * scale * scale);
        g[0] = 0.f;
#pragma unroll
        for (int i = 1; i < K; ++i) g[i] = f[i] * scale;
        S[0] = ol.a * kSqrt4Pi;
#pragma unroll
        for (int i = 1; i < K; ++i) S[i] = ol.b * g[i];
        for (int t = 0; t < k; ++t) {
            float T[K];
            sh_sqr(S, T);
#pragma unroll
            for (int i = 0; i < K; ++i) {
                hist[t][i] = S[i];
                S[i] = T[i];
            }
        }
        e0 = expf(f[0] * kInvSqrt4Pi);
#pragma unroll
        for (int i = 0; i < K; ++i) V[i] = e0 * S[i];
    }
    float H[K], ux, uy, uz, il;
    cosine_lobe(load_or(a.normals, 3 * q, live), load_or(a.normals, 3 * q + 1, live),
                load_or(a.normals, 3 * q + 2, live), H, ux, uy, uz, il);
    float W[K];
    sh_mul(V, H, W);

    // ---- shading adjoint: B_c = a_c L_c . W
    float dB[3], alb[3], loss = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        alb[c] = load_or(a.albedo, 3 * q + c, live);
        if (a.target) {
            const float r = load_or(a.radiance, 3 * q + c, live) - load_or(a.target, 3 * q + c, live);
            dB[c] = r;
            loss = fmaf(0.5f * r, r, loss);
        } else {
            dB[c] = load_or(a.d_radiance, 3 * q + c, live);
        }
    }
    float dW[K];
#pragma unroll
    for (int i = 0; i < K; ++i) dW[i] = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float u = alb[c] * dB[c];
        float lw = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const float L = s_light[c * KPAD + i];
            lw = fmaf(L, W[i], lw);
            dW[i] = fmaf(u, L, dW[i]);
        }
        if (live && a.d_albedo) a.d_albedo[3 * q + c] = dB[c] * lw;
    }
    if (a.d_light) {
        float dl[3 * K];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float u = alb[c] * dB[c];
#pragma unroll
            for (int i = 0; i < K; ++i) dl[c * K + i] = u * W[i];
        }
        warp_sum_into<3 * K>(dl, &s_dl[warp][0], lane);
    }
    if (a.target) {
        const float v = warp_sum(loss);
        if (lane == 0) s_dl[warp][3 * K] += v;
    }
    float dV[K], dH[K];
    sh_mul(dW, H, dV);                     // C is symmetric: adjoint of a*b is d*b
    sh_mul(dW, V, dH);

    // ---- normal adjoint through H = A_hat_l NORM_i Ybar_i(n / |n|)
    if (live && a.d_normals) {
        float wn[K];
#pragma unroll
        for (int i = 0; i < K; ++i) wn[i] = dH[i] * SH::ahat(band_of(i)) * SH::norm(i);
        float gx, gy, gz;
        SH::ybar_vjp(ux, uy, uz, wn, gx, gy, gz);
        const float ug = ux * gx + uy * gy + uz * gz;
        a.d_normals[3 * q] = (gx - ux * ug) * il;
        a.d_normals[3 * q + 1] = (gy - uy * ug) * il;
        a.d_normals[3 * q + 2] = (gz - uz * ug) * il;
    }

    // ---- exponential adjoint
    float dfp[K];
    if (projexp) {
        proj_exp_adjoint(f, U, dV, dfp);
    } else {
        float de0 = 0.f, dS[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            de0 = fmaf(dV[i], S[i], de0);
            dS[i] = e0 * dV[i];
        }
        for (int t = k - 1; t >= 0; --t) {
            float Ht[K], T[K];
#pragma unroll
            for (int i = 0; i < K; ++i) Ht[i] = hist[t][i];
            sh_mul(dS, Ht, T);
#pragma unroll
            for (int i = 0; i < K; ++i) dS[i] = 2.f * T[i];
        }
        // S_0 = a(s) sqrt(4 pi), S_i = b(s) g_i: dg_i = b dS_i + (dA a'/s + dB b'/s) g_i
        const float dA = dS[0] * kSqrt4Pi;
        float dB = 0.f;
#pragma unroll
        for (int i = 1; i < K; ++i) dB = fmaf(dS[i], g[i], dB);
        const float cg = fmaf(dA, ol.ca, dB * ol.cb);
        dfp[0] = de0 * e0 * kInvSqrt4Pi;
#pragma unroll
        for (int i = 1; i < K; ++i) dfp[i] = fmaf(ol.b, dS[i], cg * g[i]) * scale;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) dfp[i] *= a.sc.neg_2pi_eps * SH::norm(i);

    if constexpr (!PAIRS) {
        // split backward: the pair pass reads these coefficients
        if (live) {
#pragma unroll
            for (int i = 0; i < K; ++i) a.dfp_ws[i * P + q] = dfp[i];
        }
        return;
    }
    // ---- pair adjoints
    const bool want_sph = a.d_centers || a.d_radii;
    if (want_sph || a.d_points) {
        float gq[kMono ? SH::NG : 1];
        if constexpr (kMono) SH::grad_coeffs(dfp, gq);
        const float q0 = dfp[0];
        const Normal u{ux, uy, uz};
        float gpx = 0.f, gpy = 0.f, gpz = 0.f;
        float* my_acc = s_acc + warp * 4 * N;
        // the pair loops, instantiated with and without horizon culling so the
        // selection costs nothing per pair when it is off
        auto loops = [&](auto cull_tag) {
            constexpr bool CULL = decltype(cull_tag)::value;
            auto pair = [&](float4 sp, float& gcx, float& gcy, float& gcz, float& gr) {
                if constexpr (kMono) pair_backward_grad<CULL>(px, py, pz, sp, gq, q0, gcx, gcy, gcz, gr, u);
                else pair_backward<CULL>(px, py, pz, sp, dfp, gcx, gcy, gcz, gr, u);
            };
            if (want_sph && N >= 32) {
                // Skewed order: at step t lane l handles sphere (l + t) mod N, so the
                // 32 lanes update 32 distinct slots of the warp's accumulator row
                // with plain shared-memory read-modify-writes (no cross-lane sums).
                float4* row = reinterpret_cast<float4*>(my_acc);
                int j = lane;
#pragma unroll 1
                for (int t = 0; t < N; ++t) {
                    float gcx, gcy, gcz, gr;
                    pair(s_sph[j], gcx, gcy, gcz, gr);
                    gpx -= gcx;
                    gpy -= gcy;
                    gpz -= gcz;
                    float4 acc = row[j];
                    acc.x += gcx;
                    acc.y += gcy;
                    acc.z += gcz;
                    acc.w += gr;
                    row[j] = acc;
                    __syncwarp();
                    j = (j + 1 == N) ? 0 : j + 1;
                }
            } else {
#pragma unroll 1
                for (int j = 0; j < N; ++j) {
                    float gcx, gcy, gcz, gr;
                    pair(s_sph[j], gcx, gcy, gcz, gr);
                    gpx -= gcx;
                    gpy -= gcy;
                    gpz -= gcz;
                    if (want_sph) {
                        const float v = warp_sum4(gcx, gcy, gcz, gr, lane);
                        if ((lane & 7) == 0) my_acc[4 * j + (lane >> 3)] += v;
                    }
                }
            }
        };
        if constexpr (CULLM == 2) {
            if (a.sc.horizon_cull) loops(std::true_type{});
            else loops(std::false_type{});
        } else {
            loops(std::integral_constant<bool, CULLM == 1>{});
        }
        if (live && a.d_points) {
            a.d_points[3 * q] = gpx;
            a.d_points[3 * q + 1] = gpy;
            a.d_points[3 * q + 2] = gpz;
        }
    }
}

// The last contributor copies the accumulated scene-level sums to the
// outputs and re-zeroes the accumulator and its counter for the next launch.
__device__ void finish_scene_sums(const BwdArgs& a, int E) {
    __threadfence();
    for (int e = threadIdx.x; e < E; e += kBlock) {
        const float v = __ldcg(a.partials + e);
        a.partials[e] = 0.f;
        if (e < 3 * K) {
            if (a.d_light) a.d_light[e] = v;
        } else if (e == 3 * K) {
            if (a.loss) *a.loss = v;
        } else {
            const int s = e - (3 * K + 1), j = s >> 2, comp = s & 3;
            if (comp < 3) {
                if (a.d_centers) a.d_centers[3 * j + comp] = v;
            } else if (a.d_radii) {
                a.d_radii[j] = v;
            }
        }
    }
    if (threadIdx.x == 0) *a.counter = 0u;
}

// Layout of one block's reduced scene gradient (E floats):
//   [0, 3K)          d_light, channel-major
//   [3K]             loss
//   [3K+1, 3K+1+4N)  per sphere (d cx, d cy, d cz, d r)
// Up to 4 bands: four resident blocks per SM (<= 128 registers per thread) for
// the pair loop; above that the tail state needs the registers.
template <bool PAIRS, int CULLM, int EXPM>
__global__ void __launch_bounds__(kBlock, NB <= 4 ? SHS_BWD_MINB : SHS_BWD_MINB_HI) backward_kernel_t(BwdArgs a) {
    extern __shared__ __align__(16) float4 dyn[];
    __shared__ __align__(16) float s_light[3 * KPAD];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ float s_dl[NWARP][3 * K + 1];
    __shared__ bool s_last;
    const int N = a.sc.n_spheres;
    float4* s_sph = dyn;                  // [N]
    float* s_acc = reinterpret_cast<float*>(dyn + N);   // [NWARP][4N]
    if (!stage_scene(a.sc, s_sph, s_light, &s_bar)) return;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < NWARP * 4 * N; e += kBlock) s_acc[e] = 0.f;
    for (int e = threadIdx.x; e < NWARP * (3 * K + 1); e += kBlock) (&s_dl[0][0])[e] = 0.f;
    __syncthreads();

    const int64_t ntiles = (a.n_points + kBlock - 1) / kBlock;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
        backward_tile<PAIRS, CULLM, EXPM>(a, s_sph, s_light, s_acc, s_dl, tile, lane, warp);

    // ---- block reduction, then one scene-level reduction
    __syncthreads();
    const int E = PAIRS ? 3 * K + 1 + 4 * N : 3 * K + 1;   // tail-only: lighting and loss entries
    float* out = a.partials + static_cast<size_t>(blockIdx.x) * a.partial_stride;
    const bool det = a.counter == nullptr;
    for (int e = threadIdx.x; e < E; e += kBlock) {
        float v = 0.f;
        if (e <= 3 * K) {
#pragma unroll
            for (int w = 0; w < NWARP; ++w) v += s_dl[w][e];
        } else {
            const int s = e - (3 * K + 1);
#pragma unroll
            for (int w = 0; w < NWARP; ++w) v += s_acc[w * 4 * N + s];
        }
        if (det) out[e] = v;
        else atomicAdd(a.partials + e, v);
    }
    if (det || !PAIRS) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    finish_scene_sums(a, E);
}

// ---------------------------------------------------------------------------
// split backward, pair pass (>= 6 bands): one sphere per lane
// ---------------------------------------------------------------------------
// Work unit: 32 points.  Their gradient-polynomial coefficients (from the
// adjoint coefficients the tail pass stored) are staged in shared memory and
// read as warp-wide broadcasts; each lane owns one sphere, so sphere sums stay
// in registers and only the per-point gradient needs a cross-lane sum.
constexpr int kPtTile = 32;
// Up to 5 bands the pair pass uses the per-band gradient polynomials in
// monomial form; above that their float32 evaluation loses accuracy (large
// alternating coefficients at degree 6-7), so it uses the SH recurrences and
// their reverse sweep, broadcasting the K adjoint coefficients instead.
constexpr bool kMonoPairs = NB <= 5;
constexpr int NGP = kMonoPairs ? (SH::NG + 3) / 4 * 4 : (K + 3) / 4 * 4;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// From 7 bands the pair pass too runs four blocks per SM (8 bands: 8.8 ->
// 7.3 ms at 1M points x 300 spheres).
#if !defined(SHS_PAIRS_MINB) && SHS_NB >= 7
#define SHS_PAIRS_MINB 4
#endif
#ifdef SHS_PAIRS_MINB
#define SHS_PAIRS_BOUNDS __launch_bounds__(kBlock, SHS_PAIRS_MINB)
#else
#define SHS_PAIRS_BOUNDS __launch_bounds__(kBlock)
#endif
__global__ void SHS_PAIRS_BOUNDS bwd_pairs_t_kernel(BwdArgs a) {
    extern __shared__ __align__(16) float4 dyn[];
    __shared__ __align__(16) float s_light[3 * KPAD];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ __align__(16) float s_gq[kPtTile][NGP];
    __shared__ __align__(16) float4 s_pt[kPtTile];        // x, y, z, Phi_0
    __shared__ __align__(16) float4 s_nrm[kPtTile];       // unit normal (horizon culling)
    __shared__ float s_dpt[kPtTile][3];
    __shared__ bool s_last;
    const int N = a.sc.n_spheres;
    float4* s_sph = dyn;                                   // [N]
    float4* s_sacc = dyn + N;                              // [N] block sphere sums
    if (!stage_scene(a.sc, s_sph, s_light, &s_bar)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < N; j += kBlock) s_sacc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    const bool want_pts = a.d_points != nullptr;
    const bool cull = a.sc.horizon_cull != 0;
    const int64_t P = a.n_points;
    const int64_t nunits = (P + kPtTile - 1) / kPtTile;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        __syncthreads();
        if (tid < kPtTile) {
            const int64_t p = u * kPtTile + tid;
            const bool live = p < P;
            float dfp[K];
#pragma unroll
            for (int i = 0; i < K; ++i) dfp[i] = live ? __ldg(a.dfp_ws + i * P + p) : 0.f;
            if constexpr (kMonoPairs) {
                float gq[SH::NG];
                SH::grad_coeffs(dfp, gq);
#pragma unroll
                for (int o = 0; o < SH::NG; ++o) s_gq[tid][o] = gq[o];
            } else {
#pragma unroll
                for (int o = 0; o < K; ++o) s_gq[tid][o] = dfp[o];
            }
            s_pt[tid] = live ? make_float4(__ldg(a.points + 3 * p), __ldg(a.points + 3 * p + 1),
                                           __ldg(a.points + 3 * p + 2), dfp[0])
                             : make_float4(0.f, 0.f, 0.f, 0.f);
            if (a.sc.horizon_cull) {
                const Normal un = unit_normal(load_or(a.normals, 3 * p, live), load_or(a.normals, 3 * p + 1, live),
                                              load_or(a.normals, 3 * p + 2, live));
                s_nrm[tid] = make_float4(un.x, un.y, un.z, 0.f);
            }
            s_dpt[tid][0] = s_dpt[tid][1] = s_dpt[tid][2] = 0.f;
        }
        __syncthreads();
        for (int j0 = 0; j0 < N; j0 += kBlock) {
            if (j0 + (warp << 5) >= N) continue;   // no sphere for this warp in this round
            const int j = j0 + tid;
            const bool has = j < N;
            const float4 sp = has ? s_sph[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
            for (int t = 0; t < kPtTile; ++t) {
                const float4 pt = s_pt[t];
                float gcx, gcy, gcz, gr;
                if (cull) {
                    const float4 un = s_nrm[t];
                    const Normal u{un.x, un.y, un.z};
                    if constexpr (kMonoPairs)
                        pair_backward_grad<true>(pt.x, pt.y, pt.z, sp, &s_gq[t][0], pt.w, gcx, gcy, gcz, gr, u);
                    else
                        pair_backward<true>(pt.x, pt.y, pt.z, sp, &s_gq[t][0], gcx, gcy, gcz, gr, u);
                } else {
                    if constexpr (kMonoPairs)
                        pair_backward_grad(pt.x, pt.y, pt.z, sp, &s_gq[t][0], pt.w, gcx, gcy, gcz, gr);
                    else
                        pair_backward(pt.x, pt.y, pt.z, sp, &s_gq[t][0], gcx, gcy, gcz, gr);
                }
                if (!has) gcx = gcy = gcz = gr = 0.f;
                acc.x += gcx;
                acc.y += gcy;
                acc.z += gcz;
                acc.w += gr;
                if (want_pts) {
                    const float sx = warp_sum_f(gcx), sy = warp_sum_f(gcy), sz = warp_sum_f(gcz);
                    if (lane == 0) {
                        atomicAdd(&s_dpt[t][0], sx);
                        atomicAdd(&s_dpt[t][1], sy);
                        atomicAdd(&s_dpt[t][2], sz);
                    }
                }
            }
            if (has) {
                float4 v = s_sacc[j];
                v.x += acc.x;
                v.y += acc.y;
                v.z += acc.z;
                v.w += acc.w;
                s_sacc[j] = v;
            }
        }
        if (want_pts) {
            __syncthreads();
            if (tid < kPtTile) {
                const int64_t p = u * kPtTile + tid;
                if (p < P) {
                    a.d_points[3 * p] = -s_dpt[tid][0];
                    a.d_points[3 * p + 1] = -s_dpt[tid][1];
                    a.d_points[3 * p + 2] = -s_dpt[tid][2];
                }
            }
        }
    }
    __syncthreads();
    // sphere entries of the block's partial row (the tail pass wrote the others)
    const int E = 3 * K + 1 + 4 * N;
    float* out = a.partials + static_cast<size_t>(blockIdx.x) * a.partial_stride;
    const bool det = a.counter == nullptr;
    for (int e = 3 * K + 1 + tid; e < E; e += kBlock) {
        const int q = e - (3 * K + 1);
        const float4 v = s_sacc[q >> 2];
        const float x = (q & 3) == 0 ? v.x : (q & 3) == 1 ? v.y : (q & 3) == 2 ? v.z : v.w;
        if (det) out[e] = x;
        else atomicAdd(a.partials + e, x);
    }
    if (det) return;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    finish_scene_sums(a, E);
}

// ---------------------------------------------------------------------------
// batched persistent kernels (serving): many requests, one launch
// ---------------------------------------------------------------------------

__device__ __forceinline__ int find_request(const int64_t* tb, int n, int64_t tile) {
    int r = 0;
    while (r + 1 < n && tile >= tb[r + 1]) ++r;
    return r;
}

// Forward for every tile of every request in the batch.  Blocks take tiles
// from a device counter (consecutive tiles mostly share a request, so a
// request's scene is staged once per run of its tiles).
// SHS_BATCH_MINB_HI: minimum resident blocks of both batch kernels above 4 bands.
#ifdef SHS_BATCH_MINB_HI
#define SHS_FBATCH_BOUNDS __launch_bounds__(kBlock, NB <= 4 ? 1 : SHS_BATCH_MINB_HI)
#else
#define SHS_BATCH_MINB_HI 1
#define SHS_FBATCH_BOUNDS __launch_bounds__(kBlock)
#endif
__global__ void SHS_FBATCH_BOUNDS forward_batch_kernel(const __grid_constant__ FwdBatch b) {
    __shared__ __align__(16) float4 s_sph[kMaxSpheres];
    __shared__ __align__(16) float s_light[3 * KPAD];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ long long s_tile;
    mbar_init(&s_bar);
    int staged = -1;
    uint32_t parity = 0;
    for (;;) {
        __syncthreads();                 // previous tile done before restaging
        if (threadIdx.x == 0) s_tile = static_cast<long long>(atomicAdd(b.queue, 1u));
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= b.total_tiles) break;
        const int r = find_request(b.tile_begin, b.n, tile);
        if (r != staged) {
            if (!stage_copy(b.r[r].sc, s_sph, s_light, &s_bar, parity)) return;
            parity ^= 1u;
            staged = r;
            if constexpr (kMono) {
                interleave_sphere_pairs(s_sph, b.r[r].sc.n_spheres);
                __syncthreads();
            }
        }
        const int64_t p = (tile - b.tile_begin[r]) * kBlock + threadIdx.x;
        if (p < b.r[r].n_points) forward_point(b.r[r], s_sph, s_light, p);
    }
}

// L2 adjoint for every tile of every request in the batch.  Each tile's scene
// sums go to its request's accumulator with atomics; the tile that completes a
// request writes that request's outputs.
__global__ void __launch_bounds__(kBlock, NB <= 4 ? 4 : SHS_BATCH_MINB_HI)
    backward_batch_kernel(const __grid_constant__ BwdBatch b) {
    extern __shared__ __align__(16) float4 dyn[];
    __shared__ __align__(16) float s_light[3 * KPAD];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ float s_dl[NWARP][3 * K + 1];
    __shared__ bool s_last;
    __shared__ long long s_tile;
    float4* s_sph = dyn;                                        // [max N]
    float* s_acc = reinterpret_cast<float*>(dyn + b.max_spheres);   // [NWARP][4 max N]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    mbar_init(&s_bar);
    int staged = -1;
    uint32_t parity = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = static_cast<long long>(atomicAdd(b.queue, 1u));
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= b.total_tiles) break;
        const int r = find_request(b.tile_begin, b.n, tile);
        const BwdArgs& a = b.r[r];
        const int N = a.sc.n_spheres;
        if (r != staged) {
            if (!stage_copy(a.sc, s_sph, s_light, &s_bar, parity)) return;
            parity ^= 1u;
            staged = r;
        }
        for (int e = threadIdx.x; e < NWARP * 4 * N; e += kBlock) s_acc[e] = 0.f;
        for (int e = threadIdx.x; e < NWARP * (3 * K + 1); e += kBlock) (&s_dl[0][0])[e] = 0.f;
        __syncthreads();
        backward_tile(a, s_sph, s_light, s_acc, s_dl, tile - b.tile_begin[r], lane, warp);
        __syncthreads();
        const int E = 3 * K + 1 + 4 * N;
        for (int e = threadIdx.x; e < E; e += kBlock) {
            float v = 0.f;
            if (e <= 3 * K) {
#pragma unroll
                for (int w = 0; w < NWARP; ++w) v += s_dl[w][e];
            } else {
                const int q = e - (3 * K + 1);
#pragma unroll
                for (int w = 0; w < NWARP; ++w) v += s_acc[w * 4 * N + q];
            }
            atomicAdd(a.partials + e, v);
        }
        __threadfence();
        __syncthreads();
        const int64_t ntiles_r = b.tile_begin[r + 1] - b.tile_begin[r];
        if (threadIdx.x == 0) s_last = atomicAdd(a.counter, 1u) == static_cast<unsigned>(ntiles_r - 1);
        __syncthreads();
        if (s_last) finish_scene_sums(a, E);
    }
}

// Deterministic finish: out[e] = sum over blocks b (in order) of partials[b][e].
// One warp per 32 consecutive elements and per slice of blocks; the slices are
// then added in fixed order.
// Fixed-order sum of the blocks' partial rows.  One block per 32 entries;
// its 32 warps stride over the rows with four independent loads in flight
// each (the sum is latency-bound: ~450 rows of 32 floats per block).
constexpr int kReduceWarps = 32;

__global__ void __launch_bounds__(32 * kReduceWarps) reduce_partials_kernel(BwdArgs a, int nblk) {
    __shared__ float s[kReduceWarps][33];
    const int N = a.sc.n_spheres;
    const int E = 3 * K + 1 + 4 * N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
    if (e < E) {
        const float* col = a.partials + e;
        const size_t st = static_cast<size_t>(a.partial_stride);
        int b = warp;
        for (; b + 3 * kReduceWarps < nblk; b += 4 * kReduceWarps) {
            v0 += __ldcg(col + b * st);
            v1 += __ldcg(col + (b + kReduceWarps) * st);
            v2 += __ldcg(col + (b + 2 * kReduceWarps) * st);
            v3 += __ldcg(col + (b + 3 * kReduceWarps) * st);
        }
        for (; b < nblk; b += kReduceWarps) v0 += __ldcg(col + b * st);
    }
    s[warp][lane] = (v0 + v1) + (v2 + v3);
    __syncthreads();
    if (warp != 0 || e >= E) return;
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kReduceWarps; ++w) t += s[w][lane];
    if (e < 3 * K) {
        if (a.d_light) a.d_light[e] = t;
    } else if (e == 3 * K) {
        if (a.loss) *a.loss = t;
    } else {
        const int q = e - (3 * K + 1), j = q >> 2, comp = q & 3;
        if (comp < 3) {
            if (a.d_centers) a.d_centers[3 * j + comp] = t;
        } else if (a.d_radii) {
            a.d_radii[j] = t;
        }
    }
}

size_t backward_dyn_smem(int n_spheres) {
    return static_cast<size_t>(n_spheres) * 16u * (1 + NWARP);
}

}  // namespace

template <>
int backward_blocks_per_sm<NB>(int n_spheres) {
    cudaFuncSetAttribute(backward_kernel_t<true, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(backward_dyn_smem(kMaxSpheres)));
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, backward_kernel_t<true, 0, 0>, kBlock,
                                                      backward_dyn_smem(n_spheres)) != cudaSuccess || nb < 1)
        nb = 1;
    return nb;
}

template <>
cudaError_t launch_forward_batch<NB>(const FwdBatch& b, cudaStream_t s) {
    if (b.total_tiles <= 0) return cudaSuccess;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, forward_batch_kernel, kBlock, 0);
    if (e != cudaSuccess) return e;
    const int64_t cap = static_cast<int64_t>(sms) * (per_sm > 0 ? per_sm : 1);
    const int grid = static_cast<int>(b.total_tiles < cap ? b.total_tiles : cap);
    forward_batch_kernel<<<grid, kBlock, 0, s>>>(b);
    count_launch();
    return cudaGetLastError();
}

template <>
cudaError_t launch_backward_batch<NB>(const BwdBatch& b, cudaStream_t s) {
    if (b.total_tiles <= 0) return cudaSuccess;
    const size_t smem = backward_dyn_smem(b.max_spheres);
    static const cudaError_t attr = cudaFuncSetAttribute(
        backward_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
        static_cast<int>(backward_dyn_smem(kMaxSpheres)));
    if (attr != cudaSuccess) return attr;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, backward_batch_kernel, kBlock, smem);
    if (e != cudaSuccess) return e;
    const int64_t cap = static_cast<int64_t>(sms) * (per_sm > 0 ? per_sm : 1);
    const int grid = static_cast<int>(b.total_tiles < cap ? b.total_tiles : cap);
    backward_batch_kernel<<<grid, kBlock, smem, s>>>(b);
    count_launch();
    return cudaGetLastError();
}

template <>
cudaError_t launch_forward_pairs<NB>(const FwdArgs& a, cudaStream_t s) {
    if (a.n_points <= 0) return cudaSuccess;
    const int64_t blocks = (a.n_points + kBlock - 1) / kBlock;
    forward_kernel_t<kFwdPairs><<<static_cast<unsigned>(blocks), kBlock, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <>
cudaError_t launch_forward<NB>(const FwdArgs& a, cudaStream_t s) {
    if (a.n_points <= 0) return cudaSuccess;
    const int64_t blocks = (a.n_points + kBlock - 1) / kBlock;
    if (a.tail_only)
        forward_kernel_t<kFwdTail><<<static_cast<unsigned>(blocks), kBlock, 0, s>>>(a);
    else
        forward_kernel_t<kFwdFull><<<static_cast<unsigned>(blocks), kBlock, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template <>
cudaError_t launch_backward<NB>(const BwdArgs& a, cudaStream_t s) {
    if (a.n_points <= 0) return cudaSuccess;
    const size_t smem = backward_dyn_smem(a.sc.n_spheres);
    static const cudaError_t attr = [] {
        const int bytes = static_cast<int>(backward_dyn_smem(kMaxSpheres));
        const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaFuncSetAttribute(backward_kernel_t<true, 0, 0>, at, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(backward_kernel_t<true, 1, 0>, at, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(backward_kernel_t<true, 0, 1>, at, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(backward_kernel_t<true, 1, 1>, at, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(backward_kernel_t<true, 0, 3>, at, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(backward_kernel_t<true, 1, 3>, at, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(backward_kernel_t<false, 2, 2>, at, bytes);
        return e;
    }();
    cudaError_t err = attr;
    if (err != cudaSuccess) return err;
    if (a.dfp_ws) {
        // split backward: tail pass (per point), then the pair pass (per sphere lane)
        if (!a.skip_tail) {
            backward_kernel_t<false, 2, 2><<<static_cast<unsigned>(a.grid), kBlock, smem, s>>>(a);
            count_launch();
            err = cudaGetLastError();
            if (err != cudaSuccess) return err;
        }
        const bool need_pairs = a.d_centers || a.d_radii || a.d_points;
        static const cudaError_t attr2 = cudaFuncSetAttribute(
            bwd_pairs_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSpheres * 32);
        if (attr2 != cudaSuccess) return attr2;
        if (need_pairs || a.counter != nullptr) {
            bwd_pairs_t_kernel<<<static_cast<unsigned>(a.grid), kBlock,
                                 static_cast<size_t>(a.sc.n_spheres) * 32u, s>>>(a);
            count_launch();
            err = cudaGetLastError();
        }
    } else {
        const dim3 grid(static_cast<unsigned>(a.grid));
        if (a.sc.exp_mode == 1) {
            if (a.sc.horizon_cull) backward_kernel_t<true, 1, 1><<<grid, kBlock, smem, s>>>(a);
            else backward_kernel_t<true, 0, 1><<<grid, kBlock, smem, s>>>(a);
        } else if (a.sc.exp_mode == 2) {
            if (a.sc.horizon_cull) backward_kernel_t<true, 1, 3><<<grid, kBlock, smem, s>>>(a);
            else backward_kernel_t<true, 0, 3><<<grid, kBlock, smem, s>>>(a);
        } else {
            if (a.sc.horizon_cull) backward_kernel_t<true, 1, 0><<<grid, kBlock, smem, s>>>(a);
            else backward_kernel_t<true, 0, 0><<<grid, kBlock, smem, s>>>(a);
        }
        count_launch();
        err = cudaGetLastError();
    }
    if (err != cudaSuccess || a.counter != nullptr) return err;
    const int E = 3 * K + 1 + 4 * a.sc.n_spheres;
    reduce_partials_kernel<<<(E + 31) / 32, 32 * kReduceWarps, 0, s>>>(a, a.grid);
    count_launch();
    return cudaGetLastError();
}

}  // namespace shs
