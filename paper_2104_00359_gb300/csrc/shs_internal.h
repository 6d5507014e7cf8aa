// Internal interface between the C ABI (shs_api.cu) and the per-band-count
// kernel translation units (shs_kern.cu compiled once per n_bands).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace shs {

constexpr int kBlock = 128;          // threads per block, one shading point each
constexpr int kMaxSpheres = 1024;    // spheres staged in shared memory at once
constexpr int kMaxK = 16;            // cap on the number of squarings

// Device-side status codes (same values as shs_status).
constexpr int kDevOk = 0;
constexpr int kDevTimeout = 5;

// Scene constants a kernel needs, passed by value.
struct SceneView {
    const float4* spheres;   // [N] (cx, cy, cz, r), 16-byte aligned
    const float* light;      // [3][Kpad], Kpad = K rounded up to a multiple of 4
    int n_spheres;
    int light_stride;        // Kpad
    float neg_2pi_eps;       // -2 pi epsilon
    float tau2;              // exp_tau^2
    int kmax;
    int fixed_k;
    int horizon_cull;        // 1: drop spheres below the tangent plane, per point
    int exp_mode;            // 0: scaling + optimal linear step + squarings; 1: projected exponential;
                             // 2: as 0 with the optimal linear coefficients from a fitted table
    const float2* ol_table;  // exp_mode 2: (a, b) at the nodes s_m = m h, m = 0..ol_m-1
    int ol_m;
    float ol_inv_h;          // 1 / h
    int* status;             // device status word
};

struct FwdArgs {
    SceneView sc;
    int64_t n_points;
    const float* points;
    const float* normals;
    const float* albedo;
    float* radiance;
    float* saved_f;          // [K][P] or null
    int* saved_k;            // [P] or null
    int tail_only;           // 1: f read from saved_f (exponential and shading only)
};

struct BwdArgs {
    SceneView sc;
    int64_t n_points;
    const float* points;
    const float* normals;
    const float* albedo;
    const float* saved_f;    // [K][P] or null (recompute)
    const int* saved_k;      // [P] or null
    const float* d_radiance; // [P,3] or null when target is set
    const float* radiance;   // [P,3] (l2 mode)
    const float* target;     // [P,3] (l2 mode) or null
    float* loss;             // l2 mode
    float* d_light;
    float* d_albedo;
    float* d_centers;
    float* d_radii;
    float* d_points;
    float* d_normals;
    float* dfp_ws;           // [K][P] pair-adjoint coefficients (split backward, >= 6 bands)
    float* partials;         // [grid][stride] scratch
    unsigned int* counter;   // scratch, zero between launches
    int partial_stride;
    int grid;                // persistent grid size
    int skip_tail;           // split backward: dfp_ws and the lighting / loss rows are already written
};

// A batch: up to kMaxBatch requests (of one band count) whose 128-point tiles
// form one work list; a persistent grid pulls tiles from a device counter.
constexpr int kMaxBatch = 32;

struct FwdBatch {
    int n;
    int64_t total_tiles;
    int64_t tile_begin[kMaxBatch + 1];   // prefix sums of tiles per request
    unsigned int* queue;                  // zero before launch
    FwdArgs r[kMaxBatch];
};

struct BwdBatch {
    int n;
    int max_spheres;
    int64_t total_tiles;
    int64_t tile_begin[kMaxBatch + 1];
    unsigned int* queue;                  // zero before launch
    BwdArgs r[kMaxBatch];                 // partials/counter: per-request accumulator
};

// Reduced-precision tails on the tensor cores (8 bands): the log-visibility f
// comes from the pair pass; the tables are the quadrature's Y_c and
// (2^8 w Y)_c per chunk of directions, split into parts of the operand type
// and laid out in the canonical K-major layout, chunk after chunk.
// variant 0: the SH exponential by squarings through the 11 x 22 product rule
// (kTcQ directions); variant 1: the projected exponential, V = e0 P[exp(f^)],
// through its own 16 x 32 rule (kTcQExp directions), which also integrates
// the shading exactly.
struct TcArgs {
    SceneView sc;
    int64_t n_points;
    int prec;                // 0 = BF16 (3 parts), 1 = FP16 (2), 2 = TF32 (2)
    int variant;             // 0 = squarings, 1 = projected exponential
    const float* normals;
    const float* albedo;
    float* radiance;         // forward: [P,3] out
    const float* f;          // [K][P]
    int* saved_k;            // forward: [P] out, or null
    const void* chunks;      // tables, chunk after chunk
    const float4* dirs;      // [Q] (x, y, z, w_q); the product rule has zero weight past 242
    const float* ytab;       // [Q][64] y_i(w_q), float32
    float b2_unscale;        // 2^-8
    float lobe_c1;           // clamped-cosine lobe H(t) = c1 t + e0 + e1 t^2 + e2 t^4 + e3 t^6
    float lobe_e[4];
    // adjoint
    const int* k_in;         // [P] squarings (saved by the forward); unused by variant 1
    const float* d_radiance; // [P,3], or null in L2 mode
    const float* radiance_in;// [P,3] (L2 mode)
    const float* target;     // [P,3] (L2 mode) or null
    float* d_albedo;
    float* d_normals;
    float* dfp_ws;           // [K][P] pair-adjoint coefficients (out)
    float* partials;         // [grid][stride] lighting + loss rows, or an accumulator
    int partial_stride;
    int partial_rows;        // rows the pair pass will reduce (deterministic mode)
    int deterministic;
    float* hist;             // [grid][kMaxK][K + 2][128] squaring operands and row shifts (adjoint workspace)
};

constexpr int tc_prec_bf16 = 0, tc_prec_fp16 = 1, tc_prec_tf32 = 2;   // operand types of the tensor-core tails
constexpr int kTcQ = 256;    // product-rule directions (242 used) for 8 bands
constexpr int kTcQExp = 512; // projected-exponential rule at 8 bands: 2n x 4n = 16 x 32

template <int NB> cudaError_t launch_forward_pairs(const FwdArgs& a, cudaStream_t s);
cudaError_t launch_tail_tc_fwd(const TcArgs& a, cudaStream_t s);
cudaError_t launch_tail_tc_bwd(const TcArgs& a, cudaStream_t s);
int tail_tc_chunk(int precision, int adjoint);            // directions per table chunk (both rules)
size_t tail_tc_chunk_bytes(int precision, int adjoint);
int tail_tc_bwd_grid();                         // blocks of the adjoint tail (rows of its workspace)
template <int NB> cudaError_t launch_forward_batch(const FwdBatch& b, cudaStream_t s);
template <int NB> cudaError_t launch_backward_batch(const BwdBatch& b, cudaStream_t s);
template <int NB> cudaError_t launch_forward(const FwdArgs& a, cudaStream_t s);
template <int NB> cudaError_t launch_backward(const BwdArgs& a, cudaStream_t s);
template <int NB> int backward_blocks_per_sm(int n_spheres);
cudaError_t launch_pack_spheres(const float* centers, const float* radii, float4* out, int n,
                                bool has_c, bool has_r, cudaStream_t s);

void count_launch();

// Shared by every entry point of the C ABI (defined in shs_api.cu).
int validate_config(const void* cfg);                    // shs_status of a shs_config*
int report_error(int status, const char* fmt, ...);      // sets shs_last_error(), returns status
int report_cuda(cudaError_t e, const char* what);        // maps a CUDA error to a shs_status
cudaError_t launch_backward_nb(int n_bands, const BwdArgs& a, cudaStream_t s);
int backward_blocks_per_sm_nb(int n_bands, int n_spheres);

}  // namespace shs
