"""FP64 CPU oracle of the rasterisation step I_R = R(B(x_0..x_n), P) (Sec. 3.4,
"Rendering"): vertex radiance interpolated over a triangle mesh seen through a
4x4 projection matrix.

TEST INFRASTRUCTURE, like shs_oracle: only the tests, the package smoke check
and the benchmark's CPU legs use it.  Brute force, pixel by pixel and
triangle by triangle.

Conventions (readings; the paper uses an external rasteriser):
* clip = P [x; 1]; NDC (x, y, z) = clip_xyz / clip_w.  Pixel (r, c) of an
  H x W image has its centre at NDC x = -1 + (2c + 1) / W, y = 1 - (2r + 1) / H
  (row 0 at the top).
* A pixel shows the triangle containing its centre (screen-space barycentrics
  all >= 0, either winding) with the smallest NDC depth z in [-1, 1]; ties go
  to the lower face index.  Triangles with a vertex at clip w <= 0 are not
  drawn (no near-plane clipping).  Uncovered pixels are 0, face index -1.
* The colour is the perspective-correct interpolation
  b_k = (l_k / w_k) / sum_j (l_j / w_j) of the vertex radiance, l the
  screen-space barycentrics, w the clip w.
* Gradients: exact in the radiance; in the vertex positions through the
  barycentrics with each pixel's triangle held fixed (visibility changes carry
  no gradient).
"""

from __future__ import annotations

import numpy as np


def pixel_centres(height, width):
    """NDC (x, y) of every pixel centre, [H, W, 2]."""
    x = -1.0 + (2.0 * np.arange(width) + 1.0) / width
    y = 1.0 - (2.0 * np.arange(height) + 1.0) / height
    X, Y = np.meshgrid(x, y, indexing="xy")
    return np.stack([X, Y], axis=-1)


def project(vertices, proj):
    """Clip coordinates [V, 4] of world positions [V, 3]."""
    v = np.asarray(vertices, np.float64)
    P = np.asarray(proj, np.float64).reshape(4, 4)
    return np.concatenate([v, np.ones((v.shape[0], 1))], axis=1) @ P.T


def _edges(n0, n1, n2, q):
    """Edge functions E_k: twice the signed area of (q, and the edge opposite k)."""
    def cross(a, b, p):
        return (b[..., 0] - a[..., 0]) * (p[..., 1] - a[..., 1]) - (b[..., 1] - a[..., 1]) * (p[..., 0] - a[..., 0])
    return cross(n1, n2, q), cross(n2, n0, q), cross(n0, n1, q)


def rasterize(vertices, faces, proj, radiance, height, width):
    """Image [H, W, 3] and face index [H, W] (-1 where nothing is drawn)."""
    clip = project(vertices, proj)
    faces = np.asarray(faces, np.int64).reshape(-1, 3)
    B = np.asarray(radiance, np.float64)
    q = pixel_centres(height, width)
    best_z = np.full((height, width), np.inf)
    face_idx = np.full((height, width), -1, np.int64)
    image = np.zeros((height, width, 3))
    for f, (i0, i1, i2) in enumerate(faces):
        c = clip[[i0, i1, i2]]
        if np.any(c[:, 3] <= 0.0):
            continue
        n = c[:, :3] / c[:, 3:4]
        E = _edges(n[0], n[1], n[2], q)
        A = float(_edges(n[0], n[1], n[2], n[2])[2])      # twice the signed area = sum of the E_k
        if A == 0.0:
            continue
        lam = [e / A for e in E]
        inside = (lam[0] >= 0) & (lam[1] >= 0) & (lam[2] >= 0)
        z = lam[0] * n[0, 2] + lam[1] * n[1, 2] + lam[2] * n[2, 2]
        take = inside & (z >= -1.0) & (z <= 1.0) & (z < best_z)
        if not take.any():
            continue
        u = [lam[k] / c[k, 3] for k in range(3)]
        U = u[0] + u[1] + u[2]
        col = sum((u[k] / U)[..., None] * B[[i0, i1, i2][k]] for k in range(3))
        best_z = np.where(take, z, best_z)
        face_idx = np.where(take, f, face_idx)
        image = np.where(take[..., None], col, image)
    return image, face_idx


def shade_pixels(vertices, faces, proj, radiance, face_idx):
    """The interpolated colours for a given pixel-to-triangle assignment (the
    function whose gradient rasterize_backward returns)."""
    clip = project(vertices, proj)
    faces = np.asarray(faces, np.int64).reshape(-1, 3)
    B = np.asarray(radiance, np.float64)
    H, W = face_idx.shape
    q = pixel_centres(H, W)
    image = np.zeros((H, W, 3))
    for r in range(H):
        for cc in range(W):
            f = face_idx[r, cc]
            if f < 0:
                continue
            ids = faces[f]
            c = clip[ids]
            n = c[:, :2] / c[:, 3:4]
            E = np.array(_edges(n[0], n[1], n[2], q[r, cc]))
            u = (E / E.sum()) / c[:, 3]
            image[r, cc] = (u / u.sum()) @ B[ids]
    return image


def rasterize_backward(vertices, faces, proj, radiance, face_idx, d_image):
    """Gradients of sum(d_image * I) with respect to the vertex radiance and
    the vertex positions, each pixel's triangle held fixed."""
    clip = project(vertices, proj)
    P = np.asarray(proj, np.float64).reshape(4, 4)
    faces = np.asarray(faces, np.int64).reshape(-1, 3)
    B = np.asarray(radiance, np.float64)
    dI = np.asarray(d_image, np.float64)
    H, W = face_idx.shape
    q = pixel_centres(H, W)
    dB = np.zeros_like(B)
    dclip = np.zeros_like(clip)
    for r in range(H):
        for cc in range(W):
            f = face_idx[r, cc]
            if f < 0:
                continue
            ids = faces[f]
            c = clip[ids]
            w = c[:, 3]
            n = c[:, :2] / w[:, None]
            p = q[r, cc]
            E = np.array(_edges(n[0], n[1], n[2], p))
            A = E.sum()
            lam = E / A
            u = lam / w
            U = u.sum()
            b = u / U
            g = B[ids] @ dI[r, cc]                    # dL/db_k
            for k in range(3):
                dB[ids[k]] += b[k] * dI[r, cc]
            gam = (g - np.dot(g, b)) / U             # dL/du_k
            dlam = gam / w
            dw = -gam * lam / (w * w)
            dE = (dlam - np.dot(dlam, lam)) / A
            # E_k = cross(n_a, n_b, p) with (a, b) the edge opposite k
            dn = np.zeros((3, 2))
            for k, (a_, b_) in enumerate(((1, 2), (2, 0), (0, 1))):
                na, nb = n[a_], n[b_]
                # E = (nb.x - na.x)(p.y - na.y) - (nb.y - na.y)(p.x - na.x)
                dn[b_, 0] += dE[k] * (p[1] - na[1])
                dn[b_, 1] += -dE[k] * (p[0] - na[0])
                dn[a_, 0] += dE[k] * (-(p[1] - na[1]) + (nb[1] - na[1]))
                dn[a_, 1] += dE[k] * ((p[0] - na[0]) - (nb[0] - na[0]))
            for k in range(3):
                dclip[ids[k], 0] += dn[k, 0] / w[k]
                dclip[ids[k], 1] += dn[k, 1] / w[k]
                dclip[ids[k], 3] += dw[k] - (dn[k, 0] * n[k, 0] + dn[k, 1] * n[k, 1]) / w[k]
    d_vertices = dclip @ P[:, :3]
    return dict(d_radiance=dB, d_vertices=d_vertices)
