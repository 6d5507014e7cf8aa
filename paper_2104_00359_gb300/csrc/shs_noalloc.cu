// Backward pass that allocates no device memory (shs_shade_backward_noalloc).
//
// Some callers cannot call cudaMalloc at the point where they need gradients:
// processes whose device memory is owned by another allocator (a framework's
// caching allocator or a fixed pre-reserved pool that must account for every
// byte), and latency-critical loops that forbid allocation after start-up
// because cudaMalloc can synchronise the device.  Creating a scene allocates,
// so this entry point takes the spheres and lighting directly and keeps every
// intermediate in one statically sized device array compiled into the
// library.  The caller still provides all inputs and outputs.

#include <atomic>
#include <mutex>

#include <cuda_runtime.h>

#include "shs.h"
#include "shs_internal.h"

namespace {

// Scratch layout (floats).  Limits: n_bands <= 8 (K <= 64), n_spheres <= 1024.
constexpr int kMaxK = 64;
constexpr int kMaxN = shs::kMaxSpheres;
constexpr int kSphOff = 0;                                   // float4[kMaxN]
constexpr int kLightOff = kSphOff + 4 * kMaxN;               // [3][kMaxK]
constexpr int kAccOff = kLightOff + 3 * kMaxK + 64;          // [3K + 1 + 4N] accumulator
constexpr int kAccFloats = ((3 * kMaxK + 1 + 4 * kMaxN) + 63) / 64 * 64;
constexpr int kCounterOff = kAccOff + kAccFloats;            // unsigned counter
constexpr int kStatusOff = kCounterOff + 1;                  // int status word
constexpr int kScratchFloats = kStatusOff + 63;              // about 35 KB

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::atomic<float*> g_scratch_addr[kMaxDevices];
std::mutex g_setup_mutex;

// Device address of g_noalloc_scratch on the current device.  The host-side
// symbol is only a stand-in, so the address comes from cudaGetSymbolAddress,
// once per device, with that device current.
int scratch_for_current_device(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return shs::report_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return shs::report_error(SHS_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
    float* p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        p = g_scratch_addr[dev].load(std::memory_order_relaxed);
        if (!p) {
            void* addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess) return shs::report_cuda(e, "cudaGetSymbolAddress(no-alloc scratch)");
            p = static_cast<float*>(addr);
            g_scratch_addr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return SHS_OK;
}

}  // namespace

extern "C" shs_status shs_shade_backward_noalloc(
    const shs_config* cfg, int32_t n_spheres, const float* centers, const float* radii,
    const float* light, int64_t n_points, const float* points, const float* normals,
    const float* albedo, const void* saved, const float* d_radiance, float* d_light,
    float* d_albedo, float* d_centers, float* d_radii, float* d_points, float* d_normals,
    void* stream) {
    int st = shs::validate_config(cfg);
    if (st != SHS_OK) return static_cast<shs_status>(st);
    if (cfg->deterministic)
        return static_cast<shs_status>(shs::report_error(
            SHS_ERR_UNSUPPORTED, "no-alloc backward: deterministic sums need per-block partials, which a fixed "
                                 "array cannot hold for every grid; the sums here use atomics"));
    if (cfg->exp_mode == 2)
        return static_cast<shs_status>(shs::report_error(
            SHS_ERR_UNSUPPORTED, "no-alloc backward: exp_mode 2 needs a scene's coefficient table"));
    const int K = cfg->n_bands * cfg->n_bands;
    if (K > kMaxK)
        return static_cast<shs_status>(shs::report_error(
            SHS_ERR_INVALID_ARG, "no-alloc backward: n_bands %d exceeds its static limit of 8", cfg->n_bands));
    if (n_spheres < 0 || n_spheres > kMaxN)
        return static_cast<shs_status>(shs::report_error(
            SHS_ERR_INVALID_ARG, "no-alloc backward: n_spheres %d exceeds its static limit of %d", n_spheres, kMaxN));
    if (n_points < 0) return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "n_points < 0"));
    if (n_spheres > 0 && (!centers || !radii))
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "centers/radii are NULL"));
    if (!light) return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "light is NULL"));
    if (n_points > 0 && (!points || !normals || !albedo || !d_radiance))
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL input array"));
    if (saved && (reinterpret_cast<uintptr_t>(saved) & 15u))
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "saved not 16-byte aligned"));

    float* scratch = nullptr;
    st = scratch_for_current_device(&scratch);
    if (st != SHS_OK) return static_cast<shs_status>(st);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int Kpad = (K + 3) / 4 * 4;
    const int E = 3 * K + 1 + 4 * n_spheres;
    float4* sph = reinterpret_cast<float4*>(scratch + kSphOff);
    float* lgt = scratch + kLightOff;
    float* acc = scratch + kAccOff;
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kCounterOff);
    int* status = reinterpret_cast<int*>(scratch + kStatusOff);

    // The array keeps the previous call's contents: clear the accumulator, the
    // block counter and the status word (they must start at zero), and the
    // lighting padding.
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float) * (kStatusOff + 1 - kAccOff), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(lgt, 0, sizeof(float) * 3 * Kpad, s);
    if (e == cudaSuccess) e = cudaMemcpy2DAsync(lgt, Kpad * sizeof(float), light, K * sizeof(float),
                                                K * sizeof(float), 3, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = shs::launch_pack_spheres(centers, radii, sph, n_spheres, true, true, s);
    if (e != cudaSuccess) return static_cast<shs_status>(shs::report_cuda(e, "no-alloc backward set-up"));
    if (n_points == 0) {
        if (d_light) e = cudaMemsetAsync(d_light, 0, sizeof(float) * 3 * K, s);
        if (e == cudaSuccess && d_centers && n_spheres) e = cudaMemsetAsync(d_centers, 0, sizeof(float) * 3 * n_spheres, s);
        if (e == cudaSuccess && d_radii && n_spheres) e = cudaMemsetAsync(d_radii, 0, sizeof(float) * n_spheres, s);
        return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, "zero empty outputs"));
    }

    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return static_cast<shs_status>(shs::report_cuda(e, "query device"));

    shs::BwdArgs a{};
    a.sc.spheres = sph;
    a.sc.light = lgt;
    a.sc.n_spheres = n_spheres;
    a.sc.light_stride = Kpad;
    a.sc.neg_2pi_eps = -2.0f * 3.14159265358979323846f * cfg->epsilon;
    a.sc.tau2 = cfg->exp_tau * cfg->exp_tau;
    a.sc.kmax = cfg->exp_kmax;
    a.sc.fixed_k = cfg->fixed_k;
    a.sc.horizon_cull = cfg->horizon_cull;
    a.sc.exp_mode = cfg->exp_mode;
    a.sc.ol_table = nullptr;
    a.sc.ol_m = 0;
    a.sc.ol_inv_h = 0.f;
    a.sc.status = status;
    a.n_points = n_points;
    a.points = points;
    a.normals = normals;
    a.albedo = albedo;
    if (saved) {
        a.saved_f = static_cast<const float*>(saved);
        const size_t fbytes = (static_cast<size_t>(K) * n_points * sizeof(float) + 15) / 16 * 16;
        a.saved_k = reinterpret_cast<const int*>(static_cast<const char*>(saved) + fbytes);
    }
    a.d_radiance = d_radiance;
    a.d_light = d_light;
    a.d_albedo = d_albedo;
    a.d_centers = n_spheres ? d_centers : nullptr;
    a.d_radii = n_spheres ? d_radii : nullptr;
    a.d_points = d_points;
    a.d_normals = d_normals;
    a.partials = acc;            // one accumulator, finished by the last block
    a.counter = counter;
    a.partial_stride = E;
    const int64_t tiles = (n_points + shs::kBlock - 1) / shs::kBlock;
    const int64_t max_grid = static_cast<int64_t>(sms) * shs::backward_blocks_per_sm_nb(cfg->n_bands, n_spheres);
    a.grid = static_cast<int>(tiles < max_grid ? tiles : max_grid);
    e = shs::launch_backward_nb(cfg->n_bands, a, s);
    return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, "launch no-alloc backward"));
}

// Reads and clears the status word of the current device's array: 0, or the
// shs_status a kernel of the last no-alloc backward raised (SHS_ERR_TIMEOUT
// when a block's bounded wait for its staged spheres gave up; that call's
// scene-level sums and the failed tiles' per-point gradients were then not
// written).  Synchronises `stream`.  Allocates nothing.
extern "C" shs_status shs_noalloc_device_status(void* stream, int32_t* device_status) {
    if (!device_status) return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL argument"));
    float* scratch = nullptr;
    const int st = scratch_for_current_device(&scratch);
    if (st != SHS_OK) return static_cast<shs_status>(st);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* status = reinterpret_cast<int*>(scratch + kStatusOff);
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return static_cast<shs_status>(shs::report_cuda(e, "read no-alloc status"));
    *device_status = v;
    return SHS_OK;
}
