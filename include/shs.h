/*
 * shs.h -- C ABI of the spherical-harmonics soft-shadow shading library.
 *
 * Method: Lyu et al., "Efficient and Differentiable Shadow Computation for
 * Inverse Problems" (arXiv 2104.00359).  For every shading point x with normal
 * n and albedo a, the library evaluates
 *
 *     B_c(x) = a_c(x) * ( L_c . (V(x) * H(x)) )                  (Sec. 3.2, Eq. 8)
 *
 * where L_c are the SH lighting coefficients of colour channel c (Eq. 9),
 * H(x) is the SH projection of the clamped cosine max(n . w, 0) obtained by
 * rotating its zonal coefficients to n (Eq. 10-11), "*" is the SH triple
 * product truncated to n_bands bands (Eq. 6-7), and V(x) is the SH visibility
 * built from the sphere occluders (Sec. 3.3.2, Eq. 12-13): each sphere's
 * softened blocker (e^-epsilon inside its cap, 1 outside) contributes the
 * zonal SH of its logarithm rotated toward the sphere centre; the
 * contributions are summed and exponentiated in SH space (DC isolation,
 * scaling by 2^-k, optimal linear approximation, k squarings).
 *
 * SH basis: real orthonormal spherical harmonics without the Condon-Shortley
 * phase, linear index i = l*l + l + m (m > 0 <-> cos(m phi), m < 0 <->
 * sin(|m| phi)), K = n_bands * n_bands coefficients.  Lighting coefficients
 * passed to the library are in this basis.
 *
 * Conventions for every entry point below:
 *   - All arrays are float32, contiguous, row-major, and live in DEVICE memory
 *     (cudaMalloc or equivalent) unless a parameter says otherwise.  Pointers
 *     must be 4-byte aligned; [P,3] arrays are x,y,z triples per point.
 *   - The caller owns every array it passes.  A scene copies its spheres and
 *     lighting into device memory the library owns; they stay resident until
 *     shs_scene_destroy.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*, NULL =
 *     legacy default stream) and returns before it completes.  Calls that use
 *     the same scene must be ordered on one stream: a scene's scratch memory
 *     is shared by its calls.
 *   - Outputs are overwritten, never accumulated.  Gradients with respect to
 *     scene parameters are sums over the call's points.
 *   - Errors are returned as shs_status; no C++ exception crosses the ABI.
 *     shs_last_error() gives a thread-local message for the last failure.
 *     Invalid arguments are rejected before any work is enqueued.
 *   - NaN/Inf inputs are not checked; they propagate into the outputs.
 */
#ifndef SHS_H
#define SHS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct shs_scene_s* shs_scene_t;

typedef enum {
    SHS_OK = 0,
    SHS_ERR_INVALID_ARG = 1, /* bad size, NULL where required, out-of-range config */
    SHS_ERR_UNSUPPORTED = 2, /* valid request the library does not implement     */
    SHS_ERR_OOM = 3,         /* device allocation failed                          */
    SHS_ERR_CUDA = 4,        /* a CUDA runtime call failed (see shs_last_error)   */
    SHS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                */
    SHS_ERR_BUSY = 6         /* resource in use                                   */
} shs_status;

/* Arithmetic of the SH contractions: the squarings of the exponential (Eq. 7)
 * and the shading (Eq. 8), forward and adjoint.  The pair terms (Eq. 11-13)
 * and their adjoint, the exponent's scaling and optimal linear step always
 * run in float32.
 *   SHS_FP32: float32 on the CUDA cores (all band counts).
 *   SHS_BF16 / SHS_TF32 / SHS_FP16: tensor cores (tcgen05), n_bands = 8 only.
 *     The products run through an exact quadrature (11 x 22 directions): a
 *     squaring is X = S Y^T, S' = (X o X)(w Y), its adjoint
 *     dS = 2 ((S Y^T) o (dS' Y^T))(w Y), float32 accumulation in tensor
 *     memory.  Every operand is carried as a sum of parts of the MMA type:
 *     BF16 three parts (six MMAs per product), TF32 and FP16 two parts
 *     (three MMAs).  The shading's sums over the directions run in float32.
 *     With exp_mode 1 the projected exponential takes the same form through
 *     its 16 x 32 rule: X = f^ Y^T, U = (exp(X) o w) Y, adjoint
 *     df^ = (exp(f^ Y^T) o (dU Y^T))(w Y); BF16 and TF32 only.
 *     Error against the FP64 reference stays below 2e-3 for the radiance
 *     and every gradient output. */
enum { SHS_FP32 = 0, SHS_TF32 = 1, SHS_BF16 = 2, SHS_FP16 = 3 };

typedef struct {
    int32_t n_bands;       /* SH bands n, 1..8; K = n*n (paper uses 8, Sec. 3.2)          */
    float epsilon;         /* softened-blocker exponent, e^-eps inside a cap (Eq. 13: 3)  */
    float exp_tau;         /* scaling threshold: k = least k >= 0 with |f_hat| <= tau 2^k */
    int32_t exp_kmax;      /* cap on k, 0..16                                             */
    int32_t fixed_k;       /* >= 0: use this k for every point; < 0: per-point k          */
    int32_t precision;     /* SHS_FP32, or SHS_BF16 / SHS_TF32 / SHS_FP16 (tensor cores)  */
    int32_t deterministic; /* 1: scene gradients reduced in a fixed order                  */
    int32_t horizon_cull;  /* 0: every sphere blocks every point (Sec. 3.3.2 sums all      */
                           /*    blockers); 1: per point, skip a sphere lying entirely     */
                           /*    below the tangent plane, (c - x) . n_hat < -r (no         */
                           /*    gradient through that selection)                          */
    int32_t exp_mode;      /* 0: the SH exponential by scaling, optimal linear step and    */
                           /*    squarings (Sec. 3.3.2);  1: projected exponential         */
                           /*    P_n[exp(f)] by a 2n x 4n quadrature (FP32, or at 8 bands  */
                           /*    BF16 / TF32 on the tensor cores; FP16 is refused);        */
                           /*    2: as 0, with the optimal linear coefficients a(s), b(s)  */
                           /*    from a fitted table (shs_scene_set_ol_table)              */
} shs_config;

/* Largest node count of an optimal linear coefficient table. */
#define SHS_OL_TABLE_MAX 4096

/* Fills *cfg with n_bands=4, epsilon=3, exp_tau=1, exp_kmax=16, fixed_k=-1,
 * precision=SHS_FP32, deterministic=1, horizon_cull=0, exp_mode=0. */
shs_status shs_config_default(shs_config* cfg);

/* Creates a resident scene of n_spheres occluder spheres (Sec. 3.3.1: the
 * geometry is approximated by a sphere set) and SH lighting (Eq. 9).
 *   centers: [N,3] sphere centres, radii: [N] radii (must be >= 0; device
 *   memory, so not checked), light: [3,K] per-channel SH coefficients.
 *   0 <= n_spheres <= 1024; n_spheres == 0 is unoccluded shading, and then
 *   centers/radii may be NULL.  *out receives the handle.
 * Allocates device memory for the spheres, lighting and the scratch buffers
 * the backward pass reduces into; returns SHS_ERR_OOM if that fails. */
shs_status shs_scene_create(const shs_config* cfg, int32_t n_spheres,
                            const float* centers, const float* radii,
                            const float* light, void* stream, shs_scene_t* out);

/* Replaces centres, radii and/or lighting (NULL = unchanged) on `stream`. */
shs_status shs_scene_update(shs_scene_t scene, const float* centers,
                            const float* radii, const float* light, void* stream);

/* Optimal linear step of the SH exponential (Sec. 3.3.2, after Ren et al.'s
 * scaling / squaring setting): with g the scaled exponent (zero DC) and
 * s = |g| its coefficient norm, exp*(g) ~ a(s) sqrt(4 pi) e_0 + b(s) g.
 * exp_mode 0 uses a = b = exp(s^2 / 8 pi).  For exp_mode 2 this call sets a
 * fitted table: `table` is HOST memory [2][m], row 0 = a at the nodes
 * s_i = i s_max / (m - 1), row 1 = b; a(s), b(s) are linear between nodes
 * and constant beyond s_max.  2 <= m <= SHS_OL_TABLE_MAX, s_max > 0, every
 * entry finite (SHS_ERR_INVALID_ARG otherwise, and for a scene whose
 * exp_mode is not 2).  The call synchronises the device and copies the
 * table into scene-owned device memory; the caller keeps `table`.  Shading
 * an exp_mode 2 scene before a table is set fails with SHS_ERR_INVALID_ARG. */
shs_status shs_scene_set_ol_table(shs_scene_t scene, const float* table, int32_t m, float s_max);

/* Frees the scene after synchronising the device.  NULL is accepted. */
shs_status shs_scene_destroy(shs_scene_t scene);

/* Reads the scene's configuration and sphere count. */
shs_status shs_scene_info(shs_scene_t scene, shs_config* cfg, int32_t* n_spheres);

/* Bytes of the optional per-point state that shs_shade can save for the
 * backward pass (the log-visibility f, K floats, and the squaring count k, per
 * point).  Without it the backward pass recomputes f from the spheres. */
size_t shs_saved_bytes(shs_scene_t scene, int64_t n_points);

/* Forward shading, Eq. 8, for P = n_points points.
 *   points, normals, albedo: [P,3]; normals need not be unit length (they are
 *   normalised inside).  radiance: [P,3] output.  saved: NULL or a device
 *   buffer of shs_saved_bytes(scene, P) bytes, 16-byte aligned.
 * P == 0 is a no-op. */
shs_status shs_shade(shs_scene_t scene, int64_t n_points, const float* points,
                     const float* normals, const float* albedo, float* radiance,
                     void* saved, void* stream);

/* Shading from the saved log-visibility: the SH exponential and Eq. 8 only,
 * for a later call with the same points and spheres (the pair terms f depend
 * on geometry alone, so a lighting or albedo update, as in the paper's
 * texture and lighting optimisation (Sec. 4.1), needs no new pair pass).
 *   saved: filled by shs_shade for these points and the scene's current
 *   spheres (required); normals, albedo: [P,3]; radiance: [P,3] output.
 * The saved state is not modified. */
shs_status shs_shade_tail(shs_scene_t scene, int64_t n_points, const float* normals,
                          const float* albedo, const void* saved, float* radiance, void* stream);

/* Reverse-mode adjoint of shs_shade (Sec. 3.5: the radiance is differentiable
 * with respect to geometry, lighting and albedo).  Given d_radiance = dLoss/dB
 * [P,3], writes
 *   d_light   [3,K]  sum over points,      d_albedo  [P,3],
 *   d_centers [N,3]  sum over points,      d_radii   [N],
 *   d_points  [P,3],                       d_normals [P,3].
 * Any output pointer may be NULL to skip that gradient.  `saved` is the buffer
 * shs_shade filled for the same inputs, or NULL to recompute.  The number of
 * squarings k is piecewise constant, so no gradient flows through it; no
 * gradient flows through a clamped cap (point inside a sphere).
 * With 6 or more bands the scene keeps a workspace of K floats per point for
 * the adjoint, grown (cudaMalloc) on the first call that needs more. */
shs_status shs_shade_backward(shs_scene_t scene, int64_t n_points, const float* points,
                              const float* normals, const float* albedo, const void* saved,
                              const float* d_radiance, float* d_light, float* d_albedo,
                              float* d_centers, float* d_radii, float* d_points,
                              float* d_normals, void* stream);

/* The analysis-by-synthesis step's loss and backward pass in one launch
 * (Sec. 3.5, Eq. 15 with per-point radiance): loss = 1/2 sum (B - target)^2,
 * d_radiance = B - target, then the gradients of shs_shade_backward.
 *   radiance: [P,3] output of shs_shade for the same inputs; target: [P,3];
 *   loss: device float, written.  Other arguments as in shs_shade_backward. */
shs_status shs_shade_backward_l2(shs_scene_t scene, int64_t n_points, const float* points,
                                 const float* normals, const float* albedo, const void* saved,
                                 const float* radiance, const float* target, float* loss,
                                 float* d_light, float* d_albedo, float* d_centers,
                                 float* d_radii, float* d_points, float* d_normals,
                                 void* stream);

/* Backward pass that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * when they need gradients -- processes whose device memory belongs to another
 * allocator (a framework caching allocator or a fixed pre-reserved pool) and
 * latency-critical loops that forbid allocation after start-up.  Creating a
 * scene allocates, so it takes the spheres and lighting directly (arguments
 * as in shs_scene_create with *cfg, then as in shs_shade_backward) and keeps
 * its intermediates (packed spheres, padded lighting, the gradient
 * accumulator, a block counter and a status word) in one static device array
 * of about 35 KB compiled into the library, which every GPU that loads the
 * library holds until the process exits.
 *   Limits: n_bands <= 8 and n_spheres <= 1024; larger requests return
 *   SHS_ERR_INVALID_ARG with a message naming the limit.  exp_mode 2 (a
 *   table held by a scene) returns SHS_ERR_UNSUPPORTED.
 *   Set-up: the first call on each device looks up that array's device address
 *   (cudaGetSymbolAddress) with the device current; make that first call
 *   before any stream capture.
 *   Sharing: every call on a device uses the same array.  Each call clears
 *   the parts that must start at zero, but calls that overlap on the GPU
 *   (different streams, or different host threads) race and corrupt each
 *   other's results; order them on one stream.
 *   The scene-level sums (d_light, d_centers, d_radii) are accumulated with
 *   atomics, so their last bits can differ from run to run; cfg->deterministic
 *   = 1 returns SHS_ERR_UNSUPPORTED.
 *   Errors on the device: a block whose bounded wait for its staged spheres
 *   gives up sets a status word in the array and returns; the call then
 *   leaves d_light, d_centers, d_radii and that block's per-point gradients
 *   unwritten.  Read the word with shs_noalloc_device_status before the next
 *   call on the device (each call clears it).
 * It calls no cudaMalloc, cudaFree or allocating library routine. */
shs_status shs_shade_backward_noalloc(const shs_config* cfg, int32_t n_spheres,
                                      const float* centers, const float* radii,
                                      const float* light, int64_t n_points,
                                      const float* points, const float* normals,
                                      const float* albedo, const void* saved,
                                      const float* d_radiance, float* d_light,
                                      float* d_albedo, float* d_centers, float* d_radii,
                                      float* d_points, float* d_normals, void* stream);

/* Synchronises `stream`, then reports and clears the device-side status word
 * of shs_shade_backward_noalloc's static array on the current device: 0 = the
 * last call's kernels raised nothing, otherwise that shs_status (e.g.
 * SHS_ERR_TIMEOUT).  Allocates nothing. */
shs_status shs_noalloc_device_status(void* stream, int32_t* device_status);

/* ---- Batched shading for serving many jobs (continuous batching) ----------
 * A batch call runs the forward pass (Eq. 8) of up to 32 requests, each on its
 * own resident scene, and the L2 adjoint (as shs_shade_backward_l2) of those
 * that carry a target, in one persistent launch per band count and pass: the
 * requests' 128-point tiles form one work list that the resident blocks
 * drain through a device counter.  The paper runs one scene per call; this is
 * the serving form of the same computation (Sec. 3.5's analysis-by-synthesis
 * iterations of many jobs at once). */
typedef struct shs_batch_s* shs_batch_t;

typedef struct {
    shs_scene_t scene;      /* the job's resident scene; at most once per call  */
    int64_t n_points;       /* P >= 0                                             */
    const float* points;    /* [P,3]                                              */
    const float* normals;   /* [P,3]                                              */
    const float* albedo;    /* [P,3]                                              */
    float* radiance;        /* [P,3] output                                       */
    void* saved;            /* shs_saved_bytes(scene, P) bytes or NULL            */
    const float* target;    /* [P,3]; NULL = forward only, else L2 adjoint too    */
    float* loss;            /* adjoint outputs as in shs_shade_backward_l2,        */
    float* d_light;         /* each may be NULL                                   */
    float* d_albedo;
    float* d_centers;
    float* d_radii;
    float* d_points;
    float* d_normals;
    const float* d_radiance;/* [P,3]; with target NULL: adjoint of sum(d_radiance  */
                            /* * B) (as shs_shade_backward); radiance may then be  */
                            /* NULL, which skips the forward (saved must hold it)  */
} shs_request;

/* A batch context holds the device work counters of one in-flight batch call;
 * use one context per stream that runs batches concurrently. */
shs_status shs_batch_create(shs_batch_t* out);
shs_status shs_batch_destroy(shs_batch_t batch);

/* Enqueues the batch on `stream`.  Requests with a target or d_radiance need
 * `saved`; a request with radiance NULL and d_radiance set runs only the
 * adjoint, from the state an earlier call saved.  Two
 * requests may not share a scene (its accumulator is per call).  Scene-level
 * sums are accumulated with atomics (run-to-run rounding differences).
 * Returns SHS_ERR_INVALID_ARG for more than 32 requests. */
shs_status shs_shade_batch(shs_batch_t batch, const shs_request* reqs, int32_t n_reqs, void* stream);

/* Lighting from an environment map (Eq. 9: L_c,i = int L_c(w) y_i(w) dw),
 * for building a scene's `light` from an HDR map.
 *   env: [height][width][3] float32 device array, an equirectangular radiance
 *     map: row r covers polar angles [r, r+1] pi / height measured from +z,
 *     column c covers azimuths [c, c+1] 2 pi / width from +x toward +y
 *     (direction (sin t cos p, sin t sin p, cos t)).
 *   light: [3][K] float32 device output, K = n_bands^2, overwritten.
 *   workspace: 16-byte aligned device scratch of at least
 *     shs_envmap_workspace_bytes(height, width, n_bands) bytes (0 for invalid
 *     sizes), owned by the caller; a call uses it until it completes on
 *     `stream`, so calls that may overlap need separate workspaces.
 * Each pixel contributes its value times y_i at the pixel centre times its
 * exact solid angle (cos t_r - cos t_{r+1}) 2 pi / width.  The sum runs in a
 * fixed order (same result on every run).  1 <= height, width <= 65536 and
 * 1 <= n_bands <= 8, else SHS_ERR_INVALID_ARG, as for NULL pointers or a
 * short workspace.  Asynchronous on `stream`, except that the first call for
 * a map width on a device builds that width's azimuth table in library-owned
 * device memory (kept for later calls; up to 8 widths per device) and
 * synchronises `stream` once to do so. */
size_t shs_envmap_workspace_bytes(int32_t height, int32_t width, int32_t n_bands);
shs_status shs_project_envmap(const float* env, int32_t height, int32_t width, int32_t n_bands, float* light,
                              void* workspace, size_t workspace_bytes, void* stream);

/* Rasterisation of shaded vertices (the rendering step that follows Eq. 8:
 * I_R = R(B(x_0), ..., B(x_n), P)), with its adjoint for image-space losses.
 *   vertices: [V][3] float32 world positions, radiance: [V][3] float32 (e.g.
 *     shs_shade's output at the vertices), faces: [F][3] int32 vertex indices
 *     (device memory; a face with an index outside [0, V) is skipped).
 *   proj: 16 float32 in HOST memory, the row-major 4 x 4 matrix taking
 *     [x, y, z, 1] to clip coordinates (camera intrinsics and extrinsics).
 *   image: [height][width][3] float32 device output; face_index: [height][width]
 *     int32 device output, the triangle shown at each pixel or -1.
 *   workspace: 256-byte aligned device scratch of at least
 *     shs_raster_workspace_bytes(V, height, width) bytes, owned by the caller;
 *     calls that may overlap on the device need separate workspaces.
 * Pixel (r, c) samples NDC x = -1 + (2c + 1) / width, y = 1 - (2r + 1) / height
 * (row 0 at the top).  A pixel shows the triangle containing its centre
 * (either winding) with the smallest NDC depth in [-1, 1], ties to the lower
 * face index; triangles with a vertex at clip w <= 0 are not drawn (no
 * near-plane clipping).  Colours are perspective-correct interpolations of the
 * vertex radiance; uncovered pixels are 0.  Each triangle's thread walks its
 * pixel bounding box, so screen-filling triangles are slow.  1 <= height,
 * width <= 16384.  Asynchronous on `stream`. */
size_t shs_raster_workspace_bytes(int32_t n_vertices, int32_t height, int32_t width);
shs_status shs_rasterize(const float* vertices, int32_t n_vertices, const int32_t* faces, int32_t n_faces,
                         const float* proj, const float* radiance, int32_t height, int32_t width, float* image,
                         int32_t* face_index, void* workspace, size_t workspace_bytes, void* stream);

/* Gradients of sum(d_image * I_R) for the face_index of a shs_rasterize call
 * with the same mesh, projection and size: d_radiance [V][3] (exact) and
 * d_vertices [V][3] (through the barycentrics, each pixel's triangle held
 * fixed: visibility changes carry no gradient); both are overwritten, either
 * may be NULL.  Accumulated with atomics: rounding varies between runs. */
shs_status shs_rasterize_backward(const float* vertices, int32_t n_vertices, const int32_t* faces,
                                  int32_t n_faces, const float* proj, const float* radiance, int32_t height,
                                  int32_t width, const int32_t* face_index, const float* d_image,
                                  float* d_radiance, float* d_vertices, void* workspace, size_t workspace_bytes,
                                  void* stream);

/* ---- Scene chain: linear deformation and rigid pose (Sec. 3.3.1, 3.5) ----
 * For an array of n_rows rows (mesh vertices, normals or sphere centres):
 *   x_rest[m] = base[m] + basis[m] p,   x[m] = R(w) x_rest[m] + t
 * base [n_rows][3], basis [n_rows][3][n_params] (row-major), p [n_params],
 * pose [6] = (w, t) with R(w) = exp([w]x) (axis-angle, Rodrigues' formula);
 * direction = 1 drops t (normals).  All pointers are device memory, float32.
 * 1 <= n_params <= SHS_CHAIN_MAX_PARAMS, n_rows >= 0 (0: nothing to do).
 * Bad sizes, NULL pointers or direction outside {0, 1}: SHS_ERR_INVALID_ARG. */
#define SHS_CHAIN_MAX_PARAMS 256

/* x [n_rows][3] (and x_rest, if not NULL) on `stream`. */
shs_status shs_chain_forward(const float* base, const float* basis, int64_t n_rows, int32_t n_params,
                             const float* p, const float* pose, int32_t direction, float* x_rest, float* x,
                             void* stream);

/* Bytes of the workspace shs_chain_backward needs (0 for invalid sizes). */
size_t shs_chain_workspace_bytes(int64_t n_rows, int32_t n_params);

/* Adjoint for the upstream gradient d_x [n_rows][3]: writes (overwrites)
 *   d_p [n_params]  = sum_m basis[m]^T R^T d_x[m]
 *   d_pose [6]      = (dL/dw, dL/dt), dL/dt = sum_m d_x[m] (0 for directions),
 *                     dL/dw_a = sum_m d_x[m]^T (dR/dw_a) x_rest[m]
 * The sums are formed in a fixed order (deterministic).  workspace: device,
 * 16-byte aligned, >= shs_chain_workspace_bytes(n_rows, n_params), owned by
 * the caller and free again when the stream reaches the end of the call. */
shs_status shs_chain_backward(const float* base, const float* basis, int64_t n_rows, int32_t n_params,
                              const float* p, const float* pose, int32_t direction, const float* d_x,
                              float* d_p, float* d_pose, void* workspace, size_t workspace_bytes, void* stream);

/* The same chain for n_views rigid poses at once (the views of one mesh in a
 * multi-view optimisation): the deformation x_rest is computed once per row,
 * then each view's pose applied.  1 <= n_views <= SHS_CHAIN_MAX_VIEWS.
 *   poses [n_views][6]; x [n_views][n_rows][3] (view-major).
 * The adjoint takes d_x [n_views][n_rows][3] and writes d_p [n_params] (the
 * sum over views) and d_poses [n_views][6]; its workspace is
 * shs_chain_views_workspace_bytes(n_rows, n_params, n_views) bytes.  With
 * n_views = 1 these equal shs_chain_forward / shs_chain_backward. */
#define SHS_CHAIN_MAX_VIEWS 32
size_t shs_chain_views_workspace_bytes(int64_t n_rows, int32_t n_params, int32_t n_views);
shs_status shs_chain_forward_views(const float* base, const float* basis, int64_t n_rows, int32_t n_params,
                                   const float* p, const float* poses, int32_t n_views, int32_t direction,
                                   float* x_rest, float* x, void* stream);
shs_status shs_chain_backward_views(const float* base, const float* basis, int64_t n_rows, int32_t n_params,
                                    const float* p, const float* poses, int32_t n_views, int32_t direction,
                                    const float* d_x, float* d_p, float* d_poses, void* workspace,
                                    size_t workspace_bytes, void* stream);

/* Diagnostic: FP32 FMA throughput probe.  Launches `blocks` blocks of 256
 * threads; each thread runs 8 independent fused multiply-add chains of
 * `iters` steps (16 iters flops per thread) and writes one float to
 * out[blocks * 256] (device).  Timing it gives the measured FP32 peak that
 * the CUDA-core kernels' roofline fractions are compared with (the paper has
 * no counterpart; this is instrumentation). */
shs_status shs_fp32_fma_probe(int32_t blocks, int64_t iters, float* out, void* stream);

/* Diagnostic: one CTA computes D = A B^T with M = 128 rows, n columns and
 * inner size k on the tensor cores (tcgen05, FP32 accumulation in tensor
 * memory).  split selects the operand type: 0 = BF16; 1 = BF16 split in two
 * parts (three MMAs); 2 = BF16 in three parts (six MMAs); 3 = TF32 in two
 * parts (three MMAs); 4 = FP16 in two parts; 5-7 = as 2-4 with A held in
 * tensor memory (written there by tcgen05.st, read by the MMA) instead of
 * shared memory.  This checks the tensor-core
 * operand layouts and descriptors of the reduced-precision tails (the paper's
 * triple product, Eq. 7, and shading, Eq. 8).
 *   A: [128,k], B: [n,k], D: [128,n] float32 device arrays; 16 <= n <= 256,
 *   16 <= k <= 64, both multiples of 16 (k = 16, 32 or 64 for split >= 2).
 *   *device_status (device int) is set to SHS_ERR_TIMEOUT if the bounded wait
 *   for the MMAs gave up. */
shs_status shs_tc_gemm_selftest(const float* A, const float* B, int32_t n, int32_t k, int32_t split,
                                float* D, int32_t* device_status, void* stream);

/* Synchronises `stream`, then reports and clears the scene's device-side
 * status word: 0 = no error, otherwise a shs_status a kernel raised (e.g.
 * SHS_ERR_TIMEOUT when a bounded wait for staged data gave up). */
shs_status shs_scene_device_status(shs_scene_t scene, void* stream, int32_t* device_status);

/* Number of kernel launches the library enqueued since the process started
 * (all scenes, all threads). */
int64_t shs_launch_count(void);

const char* shs_status_string(shs_status status);
const char* shs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SHS_H */
