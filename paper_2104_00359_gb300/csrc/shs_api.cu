// C ABI of the shading library (declared in include/shs.h): argument
// validation, scene memory, and dispatch to the per-band-count kernels.

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <mutex>
#include <vector>
#include <cstdio>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "shs.h"
#include "shs_internal.h"

namespace {

thread_local char g_err[512] = "";
std::atomic<int64_t> g_launches{0};

shs_status fail(shs_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

shs_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(SHS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(SHS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

namespace shs {
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
__global__ void pack_spheres_kernel(const float* c, const float* r, float4* out, int n, bool has_c,
                                    bool has_r) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float4 v = out[j];
    if (has_c) {
        v.x = c[3 * j];
        v.y = c[3 * j + 1];
        v.z = c[3 * j + 2];
    }
    if (has_r) v.w = r[j];
    out[j] = v;
}
}  // namespace

cudaError_t launch_pack_spheres(const float* centers, const float* radii, float4* out, int n,
                                bool has_c, bool has_r, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    pack_spheres_kernel<<<(n + 127) / 128, 128, 0, s>>>(centers, radii, out, n, has_c, has_r);
    count_launch();
    return cudaGetLastError();
}
}  // namespace shs

struct shs_scene_s {
    shs_config cfg;
    int n_spheres;
    int K, Kpad;
    int device;
    int max_grid;          // persistent backward grid
    int partial_stride;    // floats per block partial
    float4* spheres;       // [max(N,1)]
    float* light;          // [3][Kpad]
    int* status;           // device status word
    float* partials;       // [max_grid][partial_stride] (deterministic) or accumulator
    unsigned int* counter;
    float* batch_acc;      // [partial_stride] accumulator for batched calls (kept zero)
    unsigned int* batch_counter;
    float* fwork;          // f storage when shs_shade gets no saved buffer (tensor-core path)
    int64_t fwork_points;
    float* bwork;          // [K][P] adjoint coefficients of the split backward (>= 6 bands)
    int64_t bwork_points;
    float* hwork;          // tensor-core adjoint: squaring operands per block [grid][kMaxK][K + 2][128]
    float2* ol_table;      // exp_mode 2: (a, b) per node
    int ol_m;
    float ol_inv_h;
};

struct shs_batch_s {
    unsigned int* queues;  // [16] tile counters: forward / backward x n_bands
};

namespace {

using shs::BwdArgs;
using shs::FwdArgs;
using shs::SceneView;

template <template <int> class F, typename... A>
cudaError_t dispatch(int nb, A&&... args) {
    switch (nb) {
        case 1: return F<1>::run(args...);
        case 2: return F<2>::run(args...);
        case 3: return F<3>::run(args...);
        case 4: return F<4>::run(args...);
        case 5: return F<5>::run(args...);
        case 6: return F<6>::run(args...);
        case 7: return F<7>::run(args...);
        case 8: return F<8>::run(args...);
        default: return cudaErrorInvalidValue;
    }
}

template <int NB> struct FwdB {
    static cudaError_t run(const shs::FwdBatch& b, cudaStream_t s) { return shs::launch_forward_batch<NB>(b, s); }
};
template <int NB> struct BwdB {
    static cudaError_t run(const shs::BwdBatch& b, cudaStream_t s) { return shs::launch_backward_batch<NB>(b, s); }
};
template <int NB> struct Fwd {
    static cudaError_t run(const FwdArgs& a, cudaStream_t s) { return shs::launch_forward<NB>(a, s); }
};
template <int NB> struct Bwd {
    static cudaError_t run(const BwdArgs& a, cudaStream_t s) { return shs::launch_backward<NB>(a, s); }
};

int blocks_per_sm(int nb, int n) {
    switch (nb) {
        case 1: return shs::backward_blocks_per_sm<1>(n);
        case 2: return shs::backward_blocks_per_sm<2>(n);
        case 3: return shs::backward_blocks_per_sm<3>(n);
        case 4: return shs::backward_blocks_per_sm<4>(n);
        case 5: return shs::backward_blocks_per_sm<5>(n);
        case 6: return shs::backward_blocks_per_sm<6>(n);
        case 7: return shs::backward_blocks_per_sm<7>(n);
        case 8: return shs::backward_blocks_per_sm<8>(n);
        default: return 1;
    }
}

shs_status check_config(const shs_config* c) {
    if (!c) return fail(SHS_ERR_INVALID_ARG, "config is NULL");
    if (c->n_bands < 1 || c->n_bands > 8) return fail(SHS_ERR_INVALID_ARG, "n_bands %d not in 1..8", c->n_bands);
    if (!(c->epsilon >= 0.f) || !(c->epsilon < 1e30f)) return fail(SHS_ERR_INVALID_ARG, "epsilon must be finite and >= 0");
    if (!(c->exp_tau > 0.f) || !(c->exp_tau < 1e30f)) return fail(SHS_ERR_INVALID_ARG, "exp_tau must be finite and > 0");
    if (c->exp_kmax < 0 || c->exp_kmax > shs::kMaxK) return fail(SHS_ERR_INVALID_ARG, "exp_kmax not in 0..%d", shs::kMaxK);
    if (c->fixed_k > shs::kMaxK) return fail(SHS_ERR_INVALID_ARG, "fixed_k > %d", shs::kMaxK);
    if (c->precision != SHS_FP32 && c->precision != SHS_TF32 && c->precision != SHS_BF16 &&
        c->precision != SHS_FP16)
        return fail(SHS_ERR_INVALID_ARG, "unknown precision %d", c->precision);
    if (c->precision != SHS_FP32 && c->n_bands != 8)
        return fail(SHS_ERR_UNSUPPORTED, "tensor-core precisions need n_bands = 8");
    if (c->deterministic != 0 && c->deterministic != 1) return fail(SHS_ERR_INVALID_ARG, "deterministic must be 0 or 1");
    if (c->horizon_cull != 0 && c->horizon_cull != 1) return fail(SHS_ERR_INVALID_ARG, "horizon_cull must be 0 or 1");
    if (c->exp_mode < 0 || c->exp_mode > 2) return fail(SHS_ERR_INVALID_ARG, "exp_mode must be 0, 1 or 2");
    if (c->exp_mode == 1 && c->precision == SHS_FP16)
        return fail(SHS_ERR_UNSUPPORTED,
                    "the projected exponential on the tensor cores takes BF16 or TF32 operands "
                    "(exp of the log-visibility exceeds the FP16 range)");
    return SHS_OK;
}

SceneView view_of(const shs_scene_s* s) {
    SceneView v;
    v.spheres = s->spheres;
    v.light = s->light;
    v.n_spheres = s->n_spheres;
    v.light_stride = s->Kpad;
    v.neg_2pi_eps = -2.0f * 3.14159265358979323846f * s->cfg.epsilon;
    v.tau2 = s->cfg.exp_tau * s->cfg.exp_tau;
    v.kmax = s->cfg.exp_kmax;
    v.fixed_k = s->cfg.fixed_k;
    v.horizon_cull = s->cfg.horizon_cull;
    v.exp_mode = s->cfg.exp_mode;
    v.ol_table = s->ol_table;
    v.ol_m = s->ol_m;
    v.ol_inv_h = s->ol_inv_h;
    v.status = s->status;
    return v;
}

bool tensor_core_precision(const shs_config& c) { return c.precision != SHS_FP32; }

// Operand type of the tensor-core tails for a shs_config precision.
int tc_prec(const shs_config& c) {
    return c.precision == SHS_TF32 ? shs::tc_prec_tf32 : c.precision == SHS_FP16 ? shs::tc_prec_fp16
                                                                                 : shs::tc_prec_bf16;
}

constexpr int kB2Shift = 8;   // power-of-two pre-scaling of w_q y_i(w_q) (keeps half-precision parts normal)

shs_status set_light(shs_scene_s* s, const float* light, cudaStream_t st) {
    cudaError_t e = cudaMemcpy2DAsync(s->light, s->Kpad * sizeof(float), light, s->K * sizeof(float),
                                      s->K * sizeof(float), 3, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SHS_OK : cuda_fail(e, "copy lighting");
}

// Real orthonormal SH (no Condon-Shortley phase) in double precision from the
// recurrences the device code uses: (x + i y)^m and d^m P_l / dz^m.
void real_sh_double(int n, double x, double y, double z, double* out) {
    double C[8], S[8], Pb[8][8];
    C[0] = 1.0;
    S[0] = 0.0;
    for (int m = 1; m < n; ++m) {
        C[m] = x * C[m - 1] - y * S[m - 1];
        S[m] = x * S[m - 1] + y * C[m - 1];
    }
    for (int m = 0; m < n; ++m) {
        double df = 1.0;
        for (int t = 1; t < 2 * m; t += 2) df *= t;
        Pb[m][m] = df;
        if (m + 1 < n) Pb[m + 1][m] = (2 * m + 1) * z * Pb[m][m];
        for (int l = m + 2; l < n; ++l)
            Pb[l][m] = ((2 * l - 1) * z * Pb[l - 1][m] - (l + m - 1) * Pb[l - 2][m]) / (l - m);
    }
    for (int l = 0; l < n; ++l) {
        for (int m = 0; m <= l; ++m) {
            double ratio = 1.0;   // (l-m)!/(l+m)!
            for (int t = l - m + 1; t <= l + m; ++t) ratio /= t;
            double N = std::sqrt((2 * l + 1) / (4.0 * M_PI) * ratio) * (m ? std::sqrt(2.0) : 1.0);
            if (m == 0) {
                out[l * l + l] = N * Pb[l][0];
            } else {
                out[l * l + l + m] = N * Pb[l][m] * C[m];
                out[l * l + l - m] = N * Pb[l][m] * S[m];
            }
        }
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method.
void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

// Tensor-core tail tables, per device, operand type and variant.  Variant 0:
// the product quadrature 11 Gauss-Legendre nodes in z x 22 uniform azimuths
// (exact for the degree-21 integrand of an 8-band triple product);
// directions 242..255 have zero weight.  Variant 1: the projected
// exponential's 2n x 4n rule, 16 x 32 (512 directions).  Built in double
// precision on the host and split there into parts of the operand type
// (p_0 = rnd(x), p_1 = rnd(x - p_0), ...).
//   chunks: per chunk c of CQ directions, the parts of Y_c (rows q, 64 columns)
//           then the parts of (2^8 w Y)_c (rows i, CQ columns), canonical
//           K-major layout;
//   dirs:   (x, y, z, w_q) per direction;  ytab: y_i(w_q) in float32.
struct TcTables {
    void* chunks = nullptr;
    float4* dirs = nullptr;
    float* ytab = nullptr;
};
TcTables g_tc_tables[64][3][2][2];   // device, operand type, forward / adjoint chunking, variant
std::mutex g_tc_mutex;

// x rounded to the operand type (round to nearest even).
double round_to(double x, int prec) {
    if (x == 0.0) return 0.0;
    int e = 0;
    std::frexp(x, &e);                                     // |x| in [2^(e-1), 2^e)
    const int bits = prec == shs::tc_prec_bf16 ? 8 : 11;   // significant bits
    // quantum: 2^(e - bits); half precision's subnormals have a fixed 2^-24
    const double q = (prec == shs::tc_prec_fp16 && e - 1 < -14) ? std::ldexp(1.0, -24) : std::ldexp(1.0, e - bits);
    return std::nearbyint(x / q) * q;
}

// Bits of a value already representable in the operand type.
uint32_t encode(double v, int prec) {
    const float f = static_cast<float>(v);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if (prec == shs::tc_prec_bf16) return u >> 16;
    if (prec == shs::tc_prec_tf32) return u;
    // IEEE half from a float that is exactly representable as one
    const uint32_t sign = (u >> 16) & 0x8000u;
    const double a = std::fabs(v);
    if (a == 0.0) return sign;
    int e = 0;
    const double m = std::frexp(a, &e);                    // a = m 2^e, m in [0.5, 1)
    if (e - 1 < -14) return sign | static_cast<uint32_t>(std::ldexp(a, 24));   // subnormal: a / 2^-24
    return sign | (static_cast<uint32_t>(e - 1 + 15) << 10) | (static_cast<uint32_t>(std::ldexp(m, 11)) & 0x3FFu);
}

// Byte offset of element (r, k) in the canonical K-major layout of an operand
// with KD columns of eb-byte elements.
size_t kmajor(int r, int k, int KD, int eb) {
    const int T = 16 / eb;
    return static_cast<size_t>(r >> 3) * (KD / T) * 128 + (k / T) * 128 + (r & 7) * 16 + (k % T) * eb;
}

void store_elem(unsigned char* base, size_t off, uint32_t bits, int eb) {
    if (eb == 2) {
        const uint16_t h = static_cast<uint16_t>(bits);
        std::memcpy(base + off, &h, 2);
    } else {
        std::memcpy(base + off, &bits, 4);
    }
}

shs_status tc_tables(int prec, int adjoint, int variant, TcTables* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(SHS_ERR_UNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lock(g_tc_mutex);
    TcTables& t = g_tc_tables[dev][prec][adjoint ? 1 : 0][variant ? 1 : 0];
    if (!t.chunks) {
        const int Q = variant ? shs::kTcQExp : shs::kTcQ, K = 64, NZ = variant ? 16 : 11, NP = variant ? 32 : 22;
        const int CQ = shs::tail_tc_chunk(prec, adjoint), NCH = Q / CQ;
        const int eb = prec == shs::tc_prec_tf32 ? 4 : 2;
        const int parts = prec == shs::tc_prec_bf16 ? 3 : 2;
        const size_t tb = static_cast<size_t>(CQ) * K * eb, chunk = 2 * parts * tb;
        if (chunk != shs::tail_tc_chunk_bytes(prec, adjoint)) return fail(SHS_ERR_UNSUPPORTED, "tensor-core chunk size");
        std::vector<double> Y(static_cast<size_t>(Q) * K, 0.0), w(Q, 0.0);
        std::vector<float4> dirs(Q, make_float4(0.f, 0.f, 0.f, 0.f));
        double zx[16], zw[16], y[64];
        gauss_legendre(NZ, zx, zw);
        for (int a = 0; a < NZ; ++a)
            for (int b = 0; b < NP; ++b) {
                const int q = a * NP + b;
                const double phi = 2.0 * M_PI * (b + 0.5) / NP, st_ = std::sqrt(1.0 - zx[a] * zx[a]);
                const double x = st_ * std::cos(phi), yy = st_ * std::sin(phi);
                real_sh_double(8, x, yy, zx[a], y);
                w[q] = zw[a] * 2.0 * M_PI / NP;
                for (int i = 0; i < K; ++i) Y[static_cast<size_t>(q) * K + i] = y[i];
                dirs[q] = make_float4(static_cast<float>(x), static_cast<float>(yy), static_cast<float>(zx[a]),
                                      static_cast<float>(w[q]));
            }
        std::vector<unsigned char> host(chunk * NCH, 0);
        std::vector<float> ytab(static_cast<size_t>(Q) * K);
        for (size_t i = 0; i < ytab.size(); ++i) ytab[i] = static_cast<float>(Y[i]);
        for (int c = 0; c < NCH; ++c) {
            unsigned char* base = host.data() + c * chunk;
            for (int r = 0; r < CQ; ++r) {
                const int q = c * CQ + r;
                for (int i = 0; i < K; ++i) {
                    double rem = Y[static_cast<size_t>(q) * K + i];
                    double rem2 = std::ldexp(w[q] * Y[static_cast<size_t>(q) * K + i], kB2Shift);
                    for (int p = 0; p < parts; ++p) {
                        const double v = round_to(rem, prec), v2 = round_to(rem2, prec);
                        rem -= v;
                        rem2 -= v2;
                        store_elem(base + p * tb, kmajor(r, i, K, eb), encode(v, prec), eb);
                        store_elem(base + (parts + p) * tb, kmajor(i, r, CQ, eb), encode(v2, prec), eb);
                    }
                }
            }
        }
        TcTables nt;
        e = cudaMalloc(&nt.chunks, host.size());
        if (e == cudaSuccess) e = cudaMalloc(&nt.dirs, sizeof(float4) * Q);
        if (e == cudaSuccess) e = cudaMalloc(&nt.ytab, sizeof(float) * Q * K);
        if (e == cudaSuccess) e = cudaMemcpy(nt.chunks, host.data(), host.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(nt.dirs, dirs.data(), sizeof(float4) * Q, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(nt.ytab, ytab.data(), sizeof(float) * Q * K, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(nt.chunks);
            cudaFree(nt.dirs);
            cudaFree(nt.ytab);
            return cuda_fail(e, "tensor-core tables");
        }
        t = nt;
    }
    *out = t;
    return SHS_OK;
}

// Clamped-cosine lobe as a polynomial in t = n . w (addition theorem):
// H(t) = sum_l A_l (2l + 1) / (4 pi) P_l(t) with A_l = 2 pi int_0^1 t P_l(t) dt,
// zero for odd l >= 3, written as c1 t + e0 + e1 t^2 + e2 t^4 + e3 t^6.
void lobe_poly(float* c1, float* e4) {
    double x[8], wt[8], c[8];
    gauss_legendre(8, x, wt);
    for (int l = 0; l < 8; ++l) {
        double s = 0.0;
        for (int g = 0; g < 8; ++g) {
            const double t = 0.5 * (x[g] + 1.0);           // [0, 1]
            double p0 = 1.0, p1 = t, pl = l == 0 ? 1.0 : t;
            for (int k = 2; k <= l; ++k) {
                pl = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = pl;
            }
            s += 0.5 * wt[g] * t * pl;
        }
        c[l] = (2 * l + 1) / 2.0 * s;                      // A_l (2l+1)/(4 pi), A_l = 2 pi s
    }
    *c1 = static_cast<float>(c[1]);
    e4[0] = static_cast<float>(c[0] - c[2] / 2 + 3 * c[4] / 8 - 5 * c[6] / 16);
    e4[1] = static_cast<float>(3 * c[2] / 2 - 30 * c[4] / 8 + 105 * c[6] / 16);
    e4[2] = static_cast<float>(35 * c[4] / 8 - 315 * c[6] / 16);
    e4[3] = static_cast<float>(231 * c[6] / 16);
}

void free_scene(shs_scene_s* s) {
    if (!s) return;
    cudaFree(s->spheres);
    cudaFree(s->light);
    cudaFree(s->status);
    cudaFree(s->partials);
    cudaFree(s->counter);
    cudaFree(s->batch_acc);
    cudaFree(s->batch_counter);
    cudaFree(s->fwork);
    cudaFree(s->bwork);
    cudaFree(s->hwork);
    cudaFree(s->ol_table);
    delete s;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool table_ready(const shs_scene_s* s) { return s->cfg.exp_mode != 2 || s->ol_table != nullptr; }

}  // namespace

namespace shs {
int validate_config(const void* cfg) { return check_config(static_cast<const shs_config*>(cfg)); }
int report_error(int status, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}
int report_cuda(cudaError_t e, const char* what) { return cuda_fail(e, what); }
cudaError_t launch_backward_nb(int n_bands, const BwdArgs& a, cudaStream_t s) {
    return dispatch<Bwd>(n_bands, a, s);
}
int backward_blocks_per_sm_nb(int n_bands, int n_spheres) { return blocks_per_sm(n_bands, n_spheres); }
}  // namespace shs

extern "C" {

shs_status shs_config_default(shs_config* cfg) {
    if (!cfg) return fail(SHS_ERR_INVALID_ARG, "config is NULL");
    cfg->n_bands = 4;
    cfg->epsilon = 3.0f;
    cfg->exp_tau = 1.0f;
    cfg->exp_kmax = 16;
    cfg->fixed_k = -1;
    cfg->precision = SHS_FP32;
    cfg->deterministic = 1;
    cfg->horizon_cull = 0;
    cfg->exp_mode = 0;
    return SHS_OK;
}

shs_status shs_scene_create(const shs_config* cfg, int32_t n_spheres, const float* centers,
                            const float* radii, const float* light, void* stream, shs_scene_t* out) {
    if (!out) return fail(SHS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    shs_status st = check_config(cfg);
    if (st != SHS_OK) return st;
    if (n_spheres < 0 || n_spheres > shs::kMaxSpheres)
        return fail(SHS_ERR_INVALID_ARG, "n_spheres %d not in 0..%d", n_spheres, shs::kMaxSpheres);
    if (n_spheres > 0 && (!centers || !radii)) return fail(SHS_ERR_INVALID_ARG, "centers/radii are NULL");
    if (!light) return fail(SHS_ERR_INVALID_ARG, "light is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    shs_scene_s* sc = new (std::nothrow) shs_scene_s();
    if (!sc) return fail(SHS_ERR_OOM, "host allocation failed");
    sc->cfg = *cfg;
    sc->n_spheres = n_spheres;
    sc->K = cfg->n_bands * cfg->n_bands;
    sc->Kpad = (sc->K + 3) / 4 * 4;
    cudaError_t e = cudaGetDevice(&sc->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sc->device);
    if (e != cudaSuccess) {
        delete sc;
        return cuda_fail(e, "query device");
    }
    sc->max_grid = sms * blocks_per_sm(cfg->n_bands, n_spheres);
    sc->partial_stride = static_cast<int>(align_up(3 * sc->K + 1 + 4 * n_spheres, 4));
    const size_t partial_floats =
        cfg->deterministic ? static_cast<size_t>(sc->max_grid) * sc->partial_stride : sc->partial_stride;
    e = cudaMalloc(&sc->spheres, sizeof(float4) * (n_spheres > 0 ? n_spheres : 1));
    if (e == cudaSuccess) e = cudaMalloc(&sc->light, sizeof(float) * 3 * sc->Kpad);
    if (e == cudaSuccess) e = cudaMalloc(&sc->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&sc->partials, sizeof(float) * partial_floats);
    if (e == cudaSuccess) e = cudaMalloc(&sc->counter, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&sc->batch_acc, sizeof(float) * sc->partial_stride);
    if (e == cudaSuccess) e = cudaMalloc(&sc->batch_counter, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->batch_acc, 0, sizeof(float) * sc->partial_stride, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->batch_counter, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->light, 0, sizeof(float) * 3 * sc->Kpad, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->partials, 0, sizeof(float) * partial_floats, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) {
        free_scene(sc);
        return cuda_fail(e, "allocate scene");
    }
    e = shs::launch_pack_spheres(centers, radii, sc->spheres, n_spheres, true, true, s);
    if (e != cudaSuccess) {
        free_scene(sc);
        return cuda_fail(e, "pack spheres");
    }
    st = set_light(sc, light, s);
    if (st != SHS_OK) {
        free_scene(sc);
        return st;
    }
    *out = sc;
    return SHS_OK;
}

shs_status shs_scene_update(shs_scene_t sc, const float* centers, const float* radii,
                            const float* light, void* stream) {
    if (!sc) return fail(SHS_ERR_INVALID_ARG, "scene is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((centers || radii) && sc->n_spheres > 0) {
        cudaError_t e = shs::launch_pack_spheres(centers, radii, sc->spheres, sc->n_spheres,
                                                 centers != nullptr, radii != nullptr, s);
        if (e != cudaSuccess) return cuda_fail(e, "pack spheres");
    }
    if (light) return set_light(sc, light, s);
    return SHS_OK;
}

shs_status shs_scene_set_ol_table(shs_scene_t sc, const float* table, int32_t m, float s_max) {
    if (!sc) return fail(SHS_ERR_INVALID_ARG, "scene is NULL");
    if (sc->cfg.exp_mode != 2) return fail(SHS_ERR_INVALID_ARG, "the scene's exp_mode is not 2");
    if (!table) return fail(SHS_ERR_INVALID_ARG, "table is NULL");
    if (m < 2 || m > SHS_OL_TABLE_MAX) return fail(SHS_ERR_INVALID_ARG, "m %d not in 2..%d", m, SHS_OL_TABLE_MAX);
    if (!(s_max > 0.f) || !(s_max < 1e30f)) return fail(SHS_ERR_INVALID_ARG, "s_max must be finite and > 0");
    std::vector<float2> ab(static_cast<size_t>(m));
    for (int i = 0; i < m; ++i) {
        const float x = table[i], y = table[m + i];
        if (!std::isfinite(x) || !std::isfinite(y)) return fail(SHS_ERR_INVALID_ARG, "table entry %d is not finite", i);
        ab[i] = make_float2(x, y);
    }
    // the previous table may still be read by queued kernels
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && sc->ol_m != m) {
        cudaFree(sc->ol_table);
        sc->ol_table = nullptr;
        sc->ol_m = 0;
        e = cudaMalloc(&sc->ol_table, sizeof(float2) * m);
    }
    if (e == cudaSuccess) e = cudaMemcpy(sc->ol_table, ab.data(), sizeof(float2) * m, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "upload coefficient table");
    sc->ol_m = m;
    sc->ol_inv_h = static_cast<float>((m - 1) / static_cast<double>(s_max));
    return SHS_OK;
}

shs_status shs_scene_destroy(shs_scene_t sc) {
    if (!sc) return SHS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_scene(sc);
    return e == cudaSuccess ? SHS_OK : cuda_fail(e, "synchronise before destroy");
}

shs_status shs_scene_info(shs_scene_t sc, shs_config* cfg, int32_t* n_spheres) {
    if (!sc) return fail(SHS_ERR_INVALID_ARG, "scene is NULL");
    if (cfg) *cfg = sc->cfg;
    if (n_spheres) *n_spheres = sc->n_spheres;
    return SHS_OK;
}

size_t shs_saved_bytes(shs_scene_t sc, int64_t n_points) {
    if (!sc || n_points <= 0) return 0;
    return align_up(static_cast<size_t>(sc->K) * n_points * sizeof(float), 16) +
           align_up(static_cast<size_t>(n_points) * sizeof(int), 16);
}

static void split_saved(shs_scene_t sc, int64_t P, void* saved, float** f, int** k) {
    if (!saved) {
        *f = nullptr;
        *k = nullptr;
        return;
    }
    *f = static_cast<float*>(saved);
    *k = reinterpret_cast<int*>(static_cast<char*>(saved) +
                                align_up(static_cast<size_t>(sc->K) * P * sizeof(float), 16));
}

shs_status shs_shade(shs_scene_t sc, int64_t n_points, const float* points, const float* normals,
                     const float* albedo, float* radiance, void* saved, void* stream) {
    if (!sc) return fail(SHS_ERR_INVALID_ARG, "scene is NULL");
    if (n_points < 0) return fail(SHS_ERR_INVALID_ARG, "n_points < 0");
    if (n_points == 0) return SHS_OK;
    if (!points || !normals || !albedo || !radiance) return fail(SHS_ERR_INVALID_ARG, "NULL input/output array");
    if (saved && (reinterpret_cast<uintptr_t>(saved) & 15u)) return fail(SHS_ERR_INVALID_ARG, "saved not 16-byte aligned");
    if (!table_ready(sc)) return fail(SHS_ERR_INVALID_ARG, "exp_mode 2 needs shs_scene_set_ol_table first");
    FwdArgs a{};
    a.sc = view_of(sc);
    a.n_points = n_points;
    a.points = points;
    a.normals = normals;
    a.albedo = albedo;
    a.radiance = radiance;
    split_saved(sc, n_points, saved, &a.saved_f, &a.saved_k);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (tensor_core_precision(sc->cfg)) {
        // pair terms in float32, then the exponential and shading on the tensor cores
        if (!a.saved_f) {
            if (sc->fwork_points < n_points) {
                cudaError_t e = cudaStreamSynchronize(st);
                cudaFree(sc->fwork);
                sc->fwork = nullptr;
                sc->fwork_points = 0;
                if (e == cudaSuccess) e = cudaMalloc(&sc->fwork, sizeof(float) * sc->K * n_points);
                if (e != cudaSuccess) return cuda_fail(e, "allocate f workspace");
                sc->fwork_points = n_points;
            }
            a.saved_f = sc->fwork;
        }
        TcTables tt;
        shs_status ts = tc_tables(tc_prec(sc->cfg), 0, sc->cfg.exp_mode == 1, &tt);
        if (ts != SHS_OK) return ts;
        cudaError_t e = shs::launch_forward_pairs<8>(a, st);
        if (e != cudaSuccess) return cuda_fail(e, "launch pair terms");
        shs::TcArgs t{};
        t.sc = a.sc;
        t.n_points = n_points;
        t.prec = tc_prec(sc->cfg);
        t.variant = sc->cfg.exp_mode == 1 ? 1 : 0;
        t.normals = normals;
        t.albedo = albedo;
        t.radiance = radiance;
        t.f = a.saved_f;
        t.saved_k = a.saved_k;
        t.chunks = tt.chunks;
        t.dirs = tt.dirs;
        t.ytab = tt.ytab;
        t.b2_unscale = std::ldexp(1.0f, -kB2Shift);
        lobe_poly(&t.lobe_c1, t.lobe_e);
        e = shs::launch_tail_tc_fwd(t, st);
        return e == cudaSuccess ? SHS_OK : cuda_fail(e, "launch tensor-core tail");
    }
    cudaError_t e = dispatch<Fwd>(sc->cfg.n_bands, a, st);
    return e == cudaSuccess ? SHS_OK : cuda_fail(e, "launch forward");
}

shs_status shs_shade_tail(shs_scene_t sc, int64_t n_points, const float* normals, const float* albedo,
                          const void* saved, float* radiance, void* stream) {
    if (!sc) return fail(SHS_ERR_INVALID_ARG, "scene is NULL");
    if (n_points < 0) return fail(SHS_ERR_INVALID_ARG, "n_points < 0");
    if (n_points == 0) return SHS_OK;
    if (!normals || !albedo || !radiance || !saved) return fail(SHS_ERR_INVALID_ARG, "NULL input/output array");
    if (reinterpret_cast<uintptr_t>(saved) & 15u) return fail(SHS_ERR_INVALID_ARG, "saved not 16-byte aligned");
    if (!table_ready(sc)) return fail(SHS_ERR_INVALID_ARG, "exp_mode 2 needs shs_scene_set_ol_table first");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* sf;
    int* sk;
    split_saved(sc, n_points, const_cast<void*>(saved), &sf, &sk);
    if (tensor_core_precision(sc->cfg)) {
        TcTables tt;
        shs_status ts = tc_tables(tc_prec(sc->cfg), 0, sc->cfg.exp_mode == 1, &tt);
        if (ts != SHS_OK) return ts;
        shs::TcArgs t{};
        t.sc = view_of(sc);
        t.n_points = n_points;
        t.prec = tc_prec(sc->cfg);
        t.variant = sc->cfg.exp_mode == 1 ? 1 : 0;
        t.normals = normals;
        t.albedo = albedo;
        t.radiance = radiance;
        t.f = sf;
        t.saved_k = nullptr;
        t.chunks = tt.chunks;
        t.dirs = tt.dirs;
        t.ytab = tt.ytab;
        t.b2_unscale = std::ldexp(1.0f, -kB2Shift);
        lobe_poly(&t.lobe_c1, t.lobe_e);
        cudaError_t e = shs::launch_tail_tc_fwd(t, st);
        return e == cudaSuccess ? SHS_OK : cuda_fail(e, "launch tensor-core tail");
    }
    FwdArgs a{};
    a.sc = view_of(sc);
    a.n_points = n_points;
    a.normals = normals;
    a.albedo = albedo;
    a.radiance = radiance;
    a.saved_f = sf;
    a.saved_k = sk;
    a.tail_only = 1;
    cudaError_t e = dispatch<Fwd>(sc->cfg.n_bands, a, st);
    return e == cudaSuccess ? SHS_OK : cuda_fail(e, "launch shading tail");
}

static shs_status backward_common(shs_scene_t sc, int64_t n_points, const float* points,
                                  const float* normals, const float* albedo, const void* saved,
                                  const float* d_radiance, const float* radiance, const float* target,
                                  float* loss, float* d_light, float* d_albedo, float* d_centers,
                                  float* d_radii, float* d_points, float* d_normals, void* stream) {
    if (!sc) return fail(SHS_ERR_INVALID_ARG, "scene is NULL");
    if (n_points < 0) return fail(SHS_ERR_INVALID_ARG, "n_points < 0");
    if (saved && (reinterpret_cast<uintptr_t>(saved) & 15u)) return fail(SHS_ERR_INVALID_ARG, "saved not 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_points == 0) {
        // empty sums: zero the scene-level outputs
        cudaError_t e = cudaSuccess;
        if (d_light) e = cudaMemsetAsync(d_light, 0, sizeof(float) * 3 * sc->K, s);
        if (e == cudaSuccess && d_centers && sc->n_spheres) e = cudaMemsetAsync(d_centers, 0, sizeof(float) * 3 * sc->n_spheres, s);
        if (e == cudaSuccess && d_radii && sc->n_spheres) e = cudaMemsetAsync(d_radii, 0, sizeof(float) * sc->n_spheres, s);
        if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
        return e == cudaSuccess ? SHS_OK : cuda_fail(e, "zero empty outputs");
    }
    if (!points || !normals || !albedo) return fail(SHS_ERR_INVALID_ARG, "NULL input array");
    if (!table_ready(sc)) return fail(SHS_ERR_INVALID_ARG, "exp_mode 2 needs shs_scene_set_ol_table first");
    BwdArgs a;
    a.sc = view_of(sc);
    a.n_points = n_points;
    a.points = points;
    a.normals = normals;
    a.albedo = albedo;
    float* sf;
    int* sk;
    split_saved(sc, n_points, const_cast<void*>(saved), &sf, &sk);
    a.saved_f = sf;
    a.saved_k = sk;
    a.d_radiance = d_radiance;
    a.radiance = radiance;
    a.target = target;
    a.loss = loss;
    a.d_light = d_light;
    a.d_albedo = d_albedo;
    a.d_centers = sc->n_spheres ? d_centers : nullptr;
    a.d_radii = sc->n_spheres ? d_radii : nullptr;
    a.d_points = d_points;
    a.d_normals = d_normals;
    a.partials = sc->partials;
    a.counter = sc->cfg.deterministic ? nullptr : sc->counter;
    a.partial_stride = sc->partial_stride;
    a.dfp_ws = nullptr;
    if (sc->cfg.n_bands >= 6) {
        // split backward: per-point tail pass, then a sphere-per-lane pair pass
        if (sc->bwork_points < n_points) {
            cudaError_t e = cudaStreamSynchronize(s);
            cudaFree(sc->bwork);
            sc->bwork = nullptr;
            sc->bwork_points = 0;
            if (e == cudaSuccess) e = cudaMalloc(&sc->bwork, sizeof(float) * sc->K * n_points);
            if (e != cudaSuccess) return cuda_fail(e, "allocate adjoint workspace");
            sc->bwork_points = n_points;
        }
        a.dfp_ws = sc->bwork;
    }
    const int64_t tiles = (n_points + shs::kBlock - 1) / shs::kBlock;
    a.grid = static_cast<int>(tiles < sc->max_grid ? tiles : sc->max_grid);
    a.skip_tail = 0;
    if (tensor_core_precision(sc->cfg)) {
        // the exponential's and the shading's adjoint on the tensor cores, then
        // the float32 pair pass of the split backward
        TcTables tt;
        shs_status ts = tc_tables(tc_prec(sc->cfg), 1, sc->cfg.exp_mode == 1, &tt);
        if (ts != SHS_OK) return ts;
        const int hgrid = shs::tail_tc_bwd_grid();
        if (!sc->hwork) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e == cudaSuccess)
                e = cudaMalloc(&sc->hwork, sizeof(float) * static_cast<size_t>(hgrid) * shs::kMaxK * (sc->K + 2) * 128);
            if (e != cudaSuccess) return cuda_fail(e, "allocate tensor-core adjoint workspace");
        }
        const float* f = sf;
        if (!f) {
            if (sc->fwork_points < n_points) {
                cudaError_t e = cudaStreamSynchronize(s);
                cudaFree(sc->fwork);
                sc->fwork = nullptr;
                sc->fwork_points = 0;
                if (e == cudaSuccess) e = cudaMalloc(&sc->fwork, sizeof(float) * sc->K * n_points);
                if (e != cudaSuccess) return cuda_fail(e, "allocate f workspace");
                sc->fwork_points = n_points;
            }
            FwdArgs fa{};
            fa.sc = a.sc;
            fa.n_points = n_points;
            fa.points = points;
            fa.normals = normals;
            fa.albedo = albedo;
            fa.radiance = nullptr;
            fa.saved_f = sc->fwork;
            fa.saved_k = nullptr;
            cudaError_t e = shs::launch_forward_pairs<8>(fa, s);
            if (e != cudaSuccess) return cuda_fail(e, "launch pair terms");
            f = sc->fwork;
        }
        shs::TcArgs t{};
        t.sc = a.sc;
        t.n_points = n_points;
        t.prec = tc_prec(sc->cfg);
        t.variant = sc->cfg.exp_mode == 1 ? 1 : 0;
        t.normals = normals;
        t.albedo = albedo;
        t.f = f;
        t.k_in = sf ? sk : nullptr;
        t.chunks = tt.chunks;
        t.dirs = tt.dirs;
        t.ytab = tt.ytab;
        t.b2_unscale = std::ldexp(1.0f, -kB2Shift);
        lobe_poly(&t.lobe_c1, t.lobe_e);
        t.d_radiance = d_radiance;
        t.radiance_in = radiance;
        t.target = target;
        t.d_albedo = d_albedo;
        t.d_normals = d_normals;
        t.dfp_ws = sc->bwork;
        t.partials = sc->partials;
        t.partial_stride = sc->partial_stride;
        t.partial_rows = a.grid;
        t.deterministic = sc->cfg.deterministic;
        t.hist = sc->hwork;
        cudaError_t e = shs::launch_tail_tc_bwd(t, s);
        if (e != cudaSuccess) return cuda_fail(e, "launch tensor-core adjoint tail");
        a.skip_tail = 1;
    }
    cudaError_t e = dispatch<Bwd>(sc->cfg.n_bands, a, s);
    return e == cudaSuccess ? SHS_OK : cuda_fail(e, "launch backward");
}

shs_status shs_shade_backward(shs_scene_t sc, int64_t n_points, const float* points,
                              const float* normals, const float* albedo, const void* saved,
                              const float* d_radiance, float* d_light, float* d_albedo,
                              float* d_centers, float* d_radii, float* d_points, float* d_normals,
                              void* stream) {
    if (n_points > 0 && !d_radiance) return fail(SHS_ERR_INVALID_ARG, "d_radiance is NULL");
    return backward_common(sc, n_points, points, normals, albedo, saved, d_radiance, nullptr, nullptr,
                           nullptr, d_light, d_albedo, d_centers, d_radii, d_points, d_normals, stream);
}

shs_status shs_shade_backward_l2(shs_scene_t sc, int64_t n_points, const float* points,
                                 const float* normals, const float* albedo, const void* saved,
                                 const float* radiance, const float* target, float* loss,
                                 float* d_light, float* d_albedo, float* d_centers, float* d_radii,
                                 float* d_points, float* d_normals, void* stream) {
    if (n_points > 0 && (!radiance || !target)) return fail(SHS_ERR_INVALID_ARG, "radiance/target is NULL");
    return backward_common(sc, n_points, points, normals, albedo, saved, nullptr, radiance, target, loss,
                           d_light, d_albedo, d_centers, d_radii, d_points, d_normals, stream);
}

shs_status shs_batch_create(shs_batch_t* out) {
    if (!out) return fail(SHS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    shs_batch_s* b = new (std::nothrow) shs_batch_s();
    if (!b) return fail(SHS_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaMalloc(&b->queues, 16 * sizeof(unsigned int));
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "allocate batch queues");
    }
    *out = b;
    return SHS_OK;
}

shs_status shs_batch_destroy(shs_batch_t b) {
    if (!b) return SHS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(b->queues);
    delete b;
    return e == cudaSuccess ? SHS_OK : cuda_fail(e, "synchronise before destroy");
}

shs_status shs_shade_batch(shs_batch_t batch, const shs_request* reqs, int32_t n_reqs, void* stream) {
    if (!batch) return fail(SHS_ERR_INVALID_ARG, "batch is NULL");
    if (n_reqs < 0 || n_reqs > shs::kMaxBatch)
        return fail(SHS_ERR_INVALID_ARG, "n_reqs %d not in 0..%d", n_reqs, shs::kMaxBatch);
    if (n_reqs > 0 && !reqs) return fail(SHS_ERR_INVALID_ARG, "reqs is NULL");
    for (int i = 0; i < n_reqs; ++i) {
        const shs_request& r = reqs[i];
        if (!r.scene) return fail(SHS_ERR_INVALID_ARG, "request %d: scene is NULL", i);
        if (!table_ready(r.scene)) return fail(SHS_ERR_INVALID_ARG, "request %d: exp_mode 2 without a table", i);
        if (r.n_points < 0) return fail(SHS_ERR_INVALID_ARG, "request %d: n_points < 0", i);
        const bool bwd_only = !r.radiance && r.d_radiance && !r.target;
        if (r.n_points > 0 && (!r.points || !r.normals || !r.albedo || (!r.radiance && !bwd_only)))
            return fail(SHS_ERR_INVALID_ARG, "request %d: NULL input/output array", i);
        if (r.target && r.d_radiance)
            return fail(SHS_ERR_INVALID_ARG, "request %d: target and d_radiance are exclusive", i);
        if ((r.target || r.d_radiance) && !r.saved)
            return fail(SHS_ERR_INVALID_ARG, "request %d: backward needs saved", i);
        if (r.saved && (reinterpret_cast<uintptr_t>(r.saved) & 15u))
            return fail(SHS_ERR_INVALID_ARG, "request %d: saved not 16-byte aligned", i);
        for (int j = 0; j < i; ++j)
            if (reqs[j].scene == r.scene)
                return fail(SHS_ERR_INVALID_ARG, "requests %d and %d share a scene", j, i);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(batch->queues, 0, 16 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(e, "reset batch queues");
    for (int nb = 1; nb <= 8 && e == cudaSuccess; ++nb) {
        shs::FwdBatch fb;
        fb.n = 0;
        fb.total_tiles = 0;
        fb.queue = batch->queues + (nb - 1);
        for (int i = 0; i < n_reqs; ++i) {
            const shs_request& r = reqs[i];
            if (r.scene->cfg.n_bands != nb || r.n_points == 0 || !r.radiance) continue;
            shs::FwdArgs& a = fb.r[fb.n];
            a = shs::FwdArgs{};
            a.sc = view_of(r.scene);
            a.n_points = r.n_points;
            a.points = r.points;
            a.normals = r.normals;
            a.albedo = r.albedo;
            a.radiance = r.radiance;
            split_saved(r.scene, r.n_points, r.saved, &a.saved_f, &a.saved_k);
            fb.tile_begin[fb.n] = fb.total_tiles;
            fb.total_tiles += (r.n_points + shs::kBlock - 1) / shs::kBlock;
            ++fb.n;
        }
        fb.tile_begin[fb.n] = fb.total_tiles;
        if (fb.n) e = dispatch<FwdB>(nb, fb, s);
    }
    for (int nb = 1; nb <= 8 && e == cudaSuccess; ++nb) {
        shs::BwdBatch bb;
        bb.n = 0;
        bb.max_spheres = 0;
        bb.total_tiles = 0;
        bb.queue = batch->queues + 8 + (nb - 1);
        for (int i = 0; i < n_reqs && e == cudaSuccess; ++i) {
            const shs_request& r = reqs[i];
            shs_scene_s* sc = r.scene;
            if (sc->cfg.n_bands != nb || (!r.target && !r.d_radiance)) continue;
            if (r.n_points == 0) {
                if (r.d_light) e = cudaMemsetAsync(r.d_light, 0, sizeof(float) * 3 * sc->K, s);
                if (e == cudaSuccess && r.d_centers && sc->n_spheres) e = cudaMemsetAsync(r.d_centers, 0, sizeof(float) * 3 * sc->n_spheres, s);
                if (e == cudaSuccess && r.d_radii && sc->n_spheres) e = cudaMemsetAsync(r.d_radii, 0, sizeof(float) * sc->n_spheres, s);
                if (e == cudaSuccess && r.loss) e = cudaMemsetAsync(r.loss, 0, sizeof(float), s);
                continue;
            }
            shs::BwdArgs& a = bb.r[bb.n];
            a = shs::BwdArgs{};
            a.sc = view_of(sc);
            a.n_points = r.n_points;
            a.points = r.points;
            a.normals = r.normals;
            a.albedo = r.albedo;
            float* sf;
            int* sk;
            split_saved(sc, r.n_points, r.saved, &sf, &sk);
            a.saved_f = sf;
            a.saved_k = sk;
            a.radiance = r.radiance;
            a.target = r.target;
            a.d_radiance = r.d_radiance;
            a.loss = r.target ? r.loss : nullptr;
            a.d_light = r.d_light;
            a.d_albedo = r.d_albedo;
            a.d_centers = sc->n_spheres ? r.d_centers : nullptr;
            a.d_radii = sc->n_spheres ? r.d_radii : nullptr;
            a.d_points = r.d_points;
            a.d_normals = r.d_normals;
            a.partials = sc->batch_acc;
            a.counter = sc->batch_counter;
            a.partial_stride = sc->partial_stride;
            bb.tile_begin[bb.n] = bb.total_tiles;
            bb.total_tiles += (r.n_points + shs::kBlock - 1) / shs::kBlock;
            if (sc->n_spheres > bb.max_spheres) bb.max_spheres = sc->n_spheres;
            ++bb.n;
        }
        bb.tile_begin[bb.n] = bb.total_tiles;
        if (e == cudaSuccess && bb.n) e = dispatch<BwdB>(nb, bb, s);
    }
    return e == cudaSuccess ? SHS_OK : cuda_fail(e, "launch batch");
}

shs_status shs_scene_device_status(shs_scene_t sc, void* stream, int32_t* device_status) {
    if (!sc || !device_status) return fail(SHS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, sc->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->status, 0, sizeof(int), s);
    if (e == cudaSuccess && v != 0) {
        // A block that gave up before adding its share left the unordered
        // accumulators part-filled and their counters short of the grid: the
        // next launch would finish early with stale sums.  Start them afresh.
        e = cudaMemsetAsync(sc->partials, 0, sizeof(float) * sc->partial_stride, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sc->counter, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sc->batch_acc, 0, sizeof(float) * sc->partial_stride, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sc->batch_counter, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "read device status");
    *device_status = v;
    return SHS_OK;
}

int64_t shs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char* shs_status_string(shs_status st) {
    switch (st) {
        case SHS_OK: return "ok";
        case SHS_ERR_INVALID_ARG: return "invalid argument";
        case SHS_ERR_UNSUPPORTED: return "unsupported";
        case SHS_ERR_OOM: return "out of device memory";
        case SHS_ERR_CUDA: return "CUDA error";
        case SHS_ERR_TIMEOUT: return "device wait timed out";
        case SHS_ERR_BUSY: return "busy";
        default: return "unknown status";
    }
}

const char* shs_last_error(void) { return g_err; }

}  // extern "C"
