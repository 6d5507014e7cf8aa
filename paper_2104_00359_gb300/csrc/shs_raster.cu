// Rasterisation of shaded vertices, I_R = R(B(x_0), ..., B(x_n), P) (the
// paper's rendering step, Sec. 3.4), and its adjoint.
//
// clip = P [x; 1], NDC = clip_xyz / clip_w.  Pixel (r, c) of an H x W image has
// its centre at NDC x = -1 + (2c + 1) / W, y = 1 - (2r + 1) / H.  A pixel shows
// the triangle that contains its centre (either winding) with the smallest
// NDC depth in [-1, 1], ties to the lower face index; triangles with a vertex
// at clip w <= 0 are not drawn.  The colour interpolates the vertex radiance
// with perspective-correct barycentrics b_k = (l_k / w_k) / sum_j l_j / w_j
// (l the screen-space barycentrics).  Gradients: exact in the radiance; in the
// vertex positions through the barycentrics, each pixel's triangle fixed.
//
// Passes: clip coordinates per vertex; per triangle, its pixel bounding box
// tested against the triangle and the (depth, face) key of each covered
// pixel folded into a 64-bit atomicMin depth buffer; per pixel, the winning
// triangle's colour.  The adjoint runs per pixel with atomic accumulation
// into per-vertex gradients (rounding order varies between runs).

#include <cstdint>
#include <cuda_runtime.h>

#include "shs.h"
#include "shs_internal.h"

namespace {

constexpr unsigned long long kEmpty = ~0ull;

struct RasterArgs {
    const float* vertices;   // [V][3]
    const int32_t* faces;    // [F][3]
    const float* radiance;   // [V][3]
    int V, F, H, W;
    float P[16];             // row-major
    float4* clip;            // [V] workspace
    unsigned long long* zbuf;   // [H*W] workspace
    float4* dclip;           // [V] workspace (adjoint)
};

__device__ __forceinline__ bool face_ids(const RasterArgs& a, int f, int& i0, int& i1, int& i2) {
    i0 = __ldg(a.faces + 3 * f);
    i1 = __ldg(a.faces + 3 * f + 1);
    i2 = __ldg(a.faces + 3 * f + 2);
    return i0 >= 0 && i1 >= 0 && i2 >= 0 && i0 < a.V && i1 < a.V && i2 < a.V;
}

// Twice the signed area of (a, b, p): the edge function of edge a -> b.
__device__ __forceinline__ float edge_fn(float ax, float ay, float bx, float by, float px, float py) {
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

// Order-preserving map of a float to uint32 (for the depth key).
__device__ __forceinline__ uint32_t ordered_bits(float z) {
    const uint32_t b = __float_as_uint(z);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void raster_clip_kernel(const __grid_constant__ RasterArgs a) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V) return;
    const float x = __ldg(a.vertices + 3 * v), y = __ldg(a.vertices + 3 * v + 1), z = __ldg(a.vertices + 3 * v + 2);
    float c[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) c[r] = fmaf(a.P[4 * r], x, fmaf(a.P[4 * r + 1], y, fmaf(a.P[4 * r + 2], z, a.P[4 * r + 3])));
    a.clip[v] = make_float4(c[0], c[1], c[2], c[3]);
}

__global__ void raster_clear_kernel(unsigned long long* zbuf, int n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) zbuf[p] = kEmpty;
}

// One thread per triangle: test the pixel centres of its bounding box.
__global__ void raster_faces_kernel(const __grid_constant__ RasterArgs a) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= a.F) return;
    int i0, i1, i2;
    if (!face_ids(a, f, i0, i1, i2)) return;
    const float4 c0 = a.clip[i0], c1 = a.clip[i1], c2 = a.clip[i2];
    if (!(c0.w > 0.f && c1.w > 0.f && c2.w > 0.f)) return;
    const float x0 = c0.x / c0.w, y0 = c0.y / c0.w, z0 = c0.z / c0.w;
    const float x1 = c1.x / c1.w, y1 = c1.y / c1.w, z1 = c1.z / c1.w;
    const float x2 = c2.x / c2.w, y2 = c2.y / c2.w, z2 = c2.z / c2.w;
    const float A = edge_fn(x0, y0, x1, y1, x2, y2);
    if (!(A != 0.f) || !isfinite(A)) return;
    const float inv_a = 1.f / A;
    // pixel ranges: column c has x = -1 + (2c + 1) / W, row r has y = 1 - (2r + 1) / H
    const float xmin = fminf(x0, fminf(x1, x2)), xmax = fmaxf(x0, fmaxf(x1, x2));
    const float ymin = fminf(y0, fminf(y1, y2)), ymax = fmaxf(y0, fmaxf(y1, y2));
    const int cmin = max(0, static_cast<int>(ceilf((xmin + 1.f) * 0.5f * a.W - 0.5f)));
    const int cmax = min(a.W - 1, static_cast<int>(floorf((xmax + 1.f) * 0.5f * a.W - 0.5f)));
    const int rmin = max(0, static_cast<int>(ceilf((1.f - ymax) * 0.5f * a.H - 0.5f)));
    const int rmax = min(a.H - 1, static_cast<int>(floorf((1.f - ymin) * 0.5f * a.H - 0.5f)));
    if (cmin > cmax || rmin > rmax) return;
    for (int r = rmin; r <= rmax; ++r) {
        const float py = 1.f - (2.f * r + 1.f) / a.H;
        for (int c = cmin; c <= cmax; ++c) {
            const float px = -1.f + (2.f * c + 1.f) / a.W;
            const float l0 = edge_fn(x1, y1, x2, y2, px, py) * inv_a;
            const float l1 = edge_fn(x2, y2, x0, y0, px, py) * inv_a;
            const float l2 = edge_fn(x0, y0, x1, y1, px, py) * inv_a;
            if (l0 < 0.f || l1 < 0.f || l2 < 0.f) continue;
            const float z = fmaf(l0, z0, fmaf(l1, z1, l2 * z2));
            if (!(z >= -1.f && z <= 1.f)) continue;
            const unsigned long long key = (static_cast<unsigned long long>(ordered_bits(z)) << 32) |
                                           static_cast<unsigned int>(f);
            atomicMin(a.zbuf + static_cast<size_t>(r) * a.W + c, key);
        }
    }
}

// Perspective-correct barycentrics of pixel (r, c) in face f; also the
// quantities the adjoint reuses.
struct PixelBary {
    float b[3], lam[3], w[3], n[3][2], U, A, px, py;
    int ids[3];
};

__device__ __forceinline__ void pixel_bary(const RasterArgs& a, int f, int r, int c, PixelBary& pb) {
    const float4 cc[3] = {a.clip[pb.ids[0]], a.clip[pb.ids[1]], a.clip[pb.ids[2]]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        pb.w[k] = cc[k].w;
        pb.n[k][0] = cc[k].x / cc[k].w;
        pb.n[k][1] = cc[k].y / cc[k].w;
    }
    pb.px = -1.f + (2.f * c + 1.f) / a.W;
    pb.py = 1.f - (2.f * r + 1.f) / a.H;
    pb.A = edge_fn(pb.n[0][0], pb.n[0][1], pb.n[1][0], pb.n[1][1], pb.n[2][0], pb.n[2][1]);
    const float inv_a = 1.f / pb.A;
    pb.lam[0] = edge_fn(pb.n[1][0], pb.n[1][1], pb.n[2][0], pb.n[2][1], pb.px, pb.py) * inv_a;
    pb.lam[1] = edge_fn(pb.n[2][0], pb.n[2][1], pb.n[0][0], pb.n[0][1], pb.px, pb.py) * inv_a;
    pb.lam[2] = edge_fn(pb.n[0][0], pb.n[0][1], pb.n[1][0], pb.n[1][1], pb.px, pb.py) * inv_a;
    float u[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = pb.lam[k] / pb.w[k];
    pb.U = u[0] + u[1] + u[2];
    const float inv_u = 1.f / pb.U;
#pragma unroll
    for (int k = 0; k < 3; ++k) pb.b[k] = u[k] * inv_u;
}

__global__ void raster_resolve_kernel(const __grid_constant__ RasterArgs a, float* image, int32_t* face_index) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.H * a.W) return;
    const unsigned long long key = a.zbuf[p];
    float col[3] = {0.f, 0.f, 0.f};
    int f = -1;
    if (key != kEmpty) {
        f = static_cast<int>(key & 0xffffffffull);
        PixelBary pb;
        face_ids(a, f, pb.ids[0], pb.ids[1], pb.ids[2]);
        pixel_bary(a, f, p / a.W, p % a.W, pb);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) col[ch] = fmaf(pb.b[k], __ldg(a.radiance + 3 * pb.ids[k] + ch), col[ch]);
    }
    image[3 * p] = col[0];
    image[3 * p + 1] = col[1];
    image[3 * p + 2] = col[2];
    face_index[p] = f;
}

// Adjoint per pixel: radiance gradients b_k dI, and the clip-coordinate
// gradients of the triangle's vertices through the barycentrics.
__global__ void raster_backward_kernel(const __grid_constant__ RasterArgs a, const int32_t* face_index,
                                       const float* d_image, float* d_radiance, int want_pos) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.H * a.W) return;
    const int f = face_index[p];
    if (f < 0 || f >= a.F) return;
    PixelBary pb;
    if (!face_ids(a, f, pb.ids[0], pb.ids[1], pb.ids[2])) return;
    pixel_bary(a, f, p / a.W, p % a.W, pb);
    const float dI[3] = {__ldg(d_image + 3 * p), __ldg(d_image + 3 * p + 1), __ldg(d_image + 3 * p + 2)};
    float g[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float* Bk = a.radiance + 3 * pb.ids[k];
        g[k] = fmaf(dI[0], __ldg(Bk), fmaf(dI[1], __ldg(Bk + 1), dI[2] * __ldg(Bk + 2)));
        if (d_radiance) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) atomicAdd(d_radiance + 3 * pb.ids[k] + ch, pb.b[k] * dI[ch]);
        }
    }
    if (!want_pos) return;
    const float bg = g[0] * pb.b[0] + g[1] * pb.b[1] + g[2] * pb.b[2];
    float dlam[3], dw[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float gam = (g[k] - bg) / pb.U;          // dL / d(l_k / w_k)
        dlam[k] = gam / pb.w[k];
        dw[k] = -gam * pb.lam[k] / (pb.w[k] * pb.w[k]);
    }
    const float ll = dlam[0] * pb.lam[0] + dlam[1] * pb.lam[1] + dlam[2] * pb.lam[2];
    float dn[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    const int ea[3] = {1, 2, 0}, eb[3] = {2, 0, 1};      // edge (a -> b) opposite vertex k
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float dE = (dlam[k] - ll) / pb.A;
        const float* na = pb.n[ea[k]];
        const float* nb = pb.n[eb[k]];
        dn[eb[k]][0] += dE * (pb.py - na[1]);
        dn[eb[k]][1] -= dE * (pb.px - na[0]);
        dn[ea[k]][0] += dE * ((nb[1] - na[1]) - (pb.py - na[1]));
        dn[ea[k]][1] += dE * ((pb.px - na[0]) - (nb[0] - na[0]));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float4* d = a.dclip + pb.ids[k];
        const float iw = 1.f / pb.w[k];
        atomicAdd(&d->x, dn[k][0] * iw);
        atomicAdd(&d->y, dn[k][1] * iw);
        atomicAdd(&d->w, dw[k] - (dn[k][0] * pb.n[k][0] + dn[k][1] * pb.n[k][1]) * iw);
    }
}

// d_vertices[v] = P[:, 0:3]^T dclip[v].
__global__ void raster_vertex_backward_kernel(const __grid_constant__ RasterArgs a, float* d_vertices) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.V) return;
    const float4 d = a.dclip[v];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        d_vertices[3 * v + j] = fmaf(d.x, a.P[j], fmaf(d.y, a.P[4 + j], fmaf(d.z, a.P[8 + j], d.w * a.P[12 + j])));
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Workspace: clip [V] float4, dclip [V] float4, depth buffer [H*W] uint64.
bool raster_setup(RasterArgs& a, const float* vertices, int32_t n_vertices, const int32_t* faces,
                  int32_t n_faces, const float* proj, const float* radiance, int32_t height, int32_t width,
                  void* workspace, size_t workspace_bytes, shs_status* st);

}  // namespace

extern "C" size_t shs_raster_workspace_bytes(int32_t n_vertices, int32_t height, int32_t width) {
    if (n_vertices < 0 || height < 1 || width < 1 || height > 16384 || width > 16384) return 0;
    const size_t v = static_cast<size_t>(n_vertices > 0 ? n_vertices : 1);
    return 2 * align256(sizeof(float4) * v) + align256(sizeof(unsigned long long) * height * width);
}

namespace {
bool raster_setup(RasterArgs& a, const float* vertices, int32_t n_vertices, const int32_t* faces,
                  int32_t n_faces, const float* proj, const float* radiance, int32_t height, int32_t width,
                  void* workspace, size_t workspace_bytes, shs_status* st) {
    auto bad = [&](const char* msg) {
        *st = static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "%s", msg));
        return false;
    };
    if (n_vertices < 0 || n_faces < 0) return bad("negative vertex or face count");
    if (height < 1 || width < 1 || height > 16384 || width > 16384) return bad("image size outside 1..16384");
    if (!proj || !workspace) return bad("NULL projection or workspace");
    if ((n_vertices > 0 && (!vertices || !radiance)) || (n_faces > 0 && !faces)) return bad("NULL mesh array");
    if (workspace_bytes < shs_raster_workspace_bytes(n_vertices, height, width)) return bad("workspace too small");
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return bad("workspace not 256-byte aligned");
    a.vertices = vertices;
    a.faces = faces;
    a.radiance = radiance;
    a.V = n_vertices;
    a.F = n_faces;
    a.H = height;
    a.W = width;
    for (int i = 0; i < 16; ++i) a.P[i] = proj[i];
    unsigned char* w = static_cast<unsigned char*>(workspace);
    const size_t vb = align256(sizeof(float4) * static_cast<size_t>(n_vertices > 0 ? n_vertices : 1));
    a.clip = reinterpret_cast<float4*>(w);
    a.dclip = reinterpret_cast<float4*>(w + vb);
    a.zbuf = reinterpret_cast<unsigned long long*>(w + 2 * vb);
    return true;
}

shs_status raster_status(cudaError_t e, const char* what) {
    return e == cudaSuccess ? SHS_OK : static_cast<shs_status>(shs::report_cuda(e, what));
}
}  // namespace

extern "C" shs_status shs_rasterize(const float* vertices, int32_t n_vertices, const int32_t* faces, int32_t n_faces,
                                    const float* proj, const float* radiance, int32_t height, int32_t width,
                                    float* image, int32_t* face_index, void* workspace, size_t workspace_bytes,
                                    void* stream) {
    RasterArgs a{};
    shs_status st = SHS_OK;
    if (!image || !face_index)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL image or face index"));
    if (!raster_setup(a, vertices, n_vertices, faces, n_faces, proj, radiance, height, width, workspace,
                      workspace_bytes, &st))
        return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int npix = height * width;
    if (n_vertices > 0) {
        raster_clip_kernel<<<(n_vertices + 255) / 256, 256, 0, s>>>(a);
        shs::count_launch();
    }
    raster_clear_kernel<<<(npix + 255) / 256, 256, 0, s>>>(a.zbuf, npix);
    shs::count_launch();
    if (n_faces > 0) {
        raster_faces_kernel<<<(n_faces + 127) / 128, 128, 0, s>>>(a);
        shs::count_launch();
    }
    raster_resolve_kernel<<<(npix + 255) / 256, 256, 0, s>>>(a, image, face_index);
    shs::count_launch();
    return raster_status(cudaGetLastError(), "rasterize");
}

extern "C" shs_status shs_rasterize_backward(const float* vertices, int32_t n_vertices, const int32_t* faces,
                                             int32_t n_faces, const float* proj, const float* radiance,
                                             int32_t height, int32_t width, const int32_t* face_index,
                                             const float* d_image, float* d_radiance, float* d_vertices,
                                             void* workspace, size_t workspace_bytes, void* stream) {
    RasterArgs a{};
    shs_status st = SHS_OK;
    if (!face_index || !d_image)
        return static_cast<shs_status>(shs::report_error(SHS_ERR_INVALID_ARG, "NULL face index or image gradient"));
    if (!raster_setup(a, vertices, n_vertices, faces, n_faces, proj, radiance, height, width, workspace,
                      workspace_bytes, &st))
        return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (n_vertices > 0) {
        if (d_radiance) e = cudaMemsetAsync(d_radiance, 0, sizeof(float) * 3 * n_vertices, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.dclip, 0, sizeof(float4) * n_vertices, s);
        if (e != cudaSuccess) return raster_status(e, "rasterize backward: clear");
        raster_clip_kernel<<<(n_vertices + 255) / 256, 256, 0, s>>>(a);
        shs::count_launch();
    }
    const int npix = height * width;
    if (n_vertices > 0 && (d_radiance || d_vertices)) {
        raster_backward_kernel<<<(npix + 255) / 256, 256, 0, s>>>(a, face_index, d_image, d_radiance,
                                                                   d_vertices ? 1 : 0);
        shs::count_launch();
        if (d_vertices) {
            raster_vertex_backward_kernel<<<(n_vertices + 255) / 256, 256, 0, s>>>(a, d_vertices);
            shs::count_launch();
        }
    }
    return raster_status(cudaGetLastError(), "rasterize backward");
}
