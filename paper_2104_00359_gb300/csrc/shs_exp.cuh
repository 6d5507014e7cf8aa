// Scaling and optimal linear step of the SH exponential (Sec. 3.3.2), shared
// by the CUDA-core kernels and the tensor-core tails.
#pragma once

#include <cuda_runtime.h>

#include "shs_internal.h"

namespace shs {
namespace {

constexpr float kSqrt4Pi = 3.5449077018110318f;
constexpr float kInvSqrt4Pi = 0.28209479177387814f;
constexpr float kInv8Pi = 0.039788735772973836f;
constexpr float kInv4Pi = 0.07957747154594767f;

// Number of squarings: least k >= 0 with |f_hat| <= tau 2^k, capped at kmax.
// Optimal linear step exp*(g) ~ a(s) sqrt(4 pi) e_0 + b(s) g at s = |g|
// (Sec. 3.3.2): the Gaussian reading a = b = exp(s^2 / 8 pi), or, for
// exp_mode 2, a fitted table that is linear between its nodes and constant
// past the last one.  ca and cb are (da/ds) / s and (db/ds) / s, the factors
// of g in the adjoint (zero at s = 0 and past the table).  TAB: Gaussian only
// (0), table only (1), or chosen by the scene's exp_mode (2).
struct OLCoef {
    float a, b, ca, cb;
};
template <int TAB = 2>
__device__ __forceinline__ OLCoef ol_coef(const SceneView& sc, float s2) {
    OLCoef r;
    if (TAB == 0 || (TAB == 2 && sc.exp_mode != 2)) {
        r.a = expf(s2 * kInv8Pi);
        r.b = r.a;
        r.ca = r.a * kInv4Pi;
        r.cb = r.ca;
        return r;
    }
    const float s = sqrtf(s2);
    const float last = static_cast<float>(sc.ol_m - 1);
    const float x = fminf(s * sc.ol_inv_h, last);
    const int i = min(static_cast<int>(x), sc.ol_m - 2);
    const float t = x - static_cast<float>(i);
    const float2 lo = __ldg(sc.ol_table + i), hi = __ldg(sc.ol_table + i + 1);
    r.a = fmaf(t, hi.x - lo.x, lo.x);
    r.b = fmaf(t, hi.y - lo.y, lo.y);
    const float c = (x < last && s > 0.f) ? sc.ol_inv_h / s : 0.f;
    r.ca = (hi.x - lo.x) * c;
    r.cb = (hi.y - lo.y) * c;
    return r;
}

__device__ __forceinline__ int scaling_k(const SceneView& sc, float nrm2) {
    if (sc.fixed_k >= 0) return sc.fixed_k;
    int k = 0;
    float thr = sc.tau2;
    while (k < sc.kmax && nrm2 > thr) {
        ++k;
        thr *= 4.f;
    }
    return k;
}

}  // namespace
}  // namespace shs
