"""Seeded synthetic scenes shaped like the paper's workloads.

The paper evaluates on meshes, HDR environment maps and reference renders that
are not distributed with it (Section 4, "Evaluation Dataset").  These
generators stand in for them: every array is drawn from
``numpy.random.default_rng(seed)`` in float64 and rounded to float32, so the
CUDA path and the FP64 oracle consume bit-identical inputs.

This module holds scene construction only (grids, capsule chains, height
fields, random draws).  It contains none of the shading method's arithmetic:
no spherical harmonics, no visibility, no exponentials.  It is the one module
that both the oracle-based tests and the CUDA path import.

Every generator returns a ``dict`` with float32 numpy arrays:

* ``points``  [P, 3]  shading-point positions
* ``normals`` [P, 3]  unit normals
* ``albedo``  [P, 3]  diffuse albedo per colour channel
* ``centers`` [N, 3]  sphere centres
* ``radii``   [N]     sphere radii
* ``light``   [3, K]  SH lighting per colour channel, K = n_bands**2
* ``n_bands`` int
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "plane_grid_scene",
    "capsule_body_scene",
    "height_field_scene",
    "random_scene",
    "perturb_scene",
    "sh_lighting",
    "serving_job",
    "mesh_deformation_scene",
    "environment_map",
    "uv_grid_faces",
    "look_at_perspective",
]


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def sh_lighting(rng, n_bands, sigma=0.3, dc=1.0, band_decay=False):
    """Per-channel SH lighting coefficients [3, K]: N(0, sigma) with the l=0
    term set to ``dc``.  With ``band_decay`` the band-l coefficients are
    divided by (l + 1)."""
    K = n_bands * n_bands
    L = rng.normal(0.0, sigma, size=(3, K))
    if band_decay:
        band = np.floor(np.sqrt(np.arange(K))).astype(np.int64)
        L = L / (band + 1.0)[None, :]
    L[:, 0] = dc
    return L


def plane_grid_scene(seed=0, grid=32, n_spheres=8, n_bands=4):
    """Plane z=0 over [-1,1]^2 sampled at ``grid`` x ``grid`` pixel centres,
    normals (0,0,1), albedo 0.5; sphere centres uniform in
    [-0.8,0.8]^2 x [0.1,0.6], radii uniform in [0.05,0.2]; lighting N(0,0.3)
    per channel with l=0 term 1.0.  Draw order: centres, radii, lighting."""
    rng = np.random.default_rng(seed)
    t = -1.0 + (2.0 * np.arange(grid) + 1.0) / grid
    X, Y = np.meshgrid(t, t, indexing="xy")
    P = grid * grid
    points = np.stack([X.ravel(), Y.ravel(), np.zeros(P)], axis=1)
    normals = np.tile([0.0, 0.0, 1.0], (P, 1))
    albedo = np.full((P, 3), 0.5)
    lo = np.array([-0.8, -0.8, 0.1])
    hi = np.array([0.8, 0.8, 0.6])
    centers = lo + (hi - lo) * rng.random((n_spheres, 3))
    radii = rng.uniform(0.05, 0.2, size=n_spheres)
    light = sh_lighting(rng, n_bands)
    return dict(points=_f32(points), normals=_f32(normals), albedo=_f32(albedo),
                centers=_f32(centers), radii=_f32(radii), light=_f32(light),
                n_bands=n_bands)


def _bone_chain(rng, n_bones, lo, hi, step=(0.12, 0.22)):
    """Random-walk joint chain kept inside the box [lo, hi] by reflection."""
    joints = [lo + (hi - lo) * (0.3 + 0.4 * rng.random(3))]
    for _ in range(n_bones):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        nxt = joints[-1] + d * rng.uniform(*step)
        nxt = np.where(nxt < lo, 2 * lo - nxt, nxt)
        nxt = np.where(nxt > hi, 2 * hi - nxt, nxt)
        joints.append(nxt)
    return np.array(joints)


def capsule_body_scene(seed=1, res=512, n_bones=20, spheres_per_bone=5,
                       n_bands=4, capsule_samples=24):
    """Human-scale G-buffer: an orthographic top-down ``res`` x ``res`` depth
    map over [-1,1]^2 of a 20-bone random-walk chain of capsules whose joints
    lie in a 2 m box and stay at least 0.15 above the ground plane z=0.

    Each bone carries ``spheres_per_bone`` occluder spheres evenly spaced on
    its axis (radii uniform in [0.02, 0.12]); the capsule radius is the
    largest of them plus 0.01.  The capsule surface is taken as the union of
    ``capsule_samples`` spheres of that radius along the axis, so each pixel's
    first hit and unit normal are analytic ray-sphere results.  Pixels that
    miss the body hit the ground plane (normal +z).  Albedo is uniform in
    [0.2, 0.9] per channel.  Lighting: N(0,0.3), l=0 term 1.0.
    """
    rng = np.random.default_rng(seed)
    lo = np.array([-0.85, -0.85, 0.15 + 0.13])
    hi = np.array([0.85, 0.85, 1.6])
    joints = _bone_chain(rng, n_bones, lo, hi)
    ts = (np.arange(spheres_per_bone) + 0.5) / spheres_per_bone
    centers, radii, cap_r = [], [], []
    for b in range(n_bones):
        a, e = joints[b], joints[b + 1]
        r = rng.uniform(0.02, 0.12, size=spheres_per_bone)
        for t, ri in zip(ts, r):
            centers.append(a + t * (e - a))
            radii.append(ri)
        cap_r.append(r.max() + 0.01)
    centers = np.array(centers)
    radii = np.array(radii)

    t = -1.0 + (2.0 * np.arange(res) + 1.0) / res
    X, Y = np.meshgrid(t, t, indexing="xy")
    X = X.ravel()
    Y = Y.ravel()
    P = X.size
    zbest = np.zeros(P)
    nrm = np.tile([0.0, 0.0, 1.0], (P, 1))
    us = np.linspace(0.0, 1.0, capsule_samples)
    for b in range(n_bones):
        a, e, R = joints[b], joints[b + 1], cap_r[b]
        for u in us:
            c = a + u * (e - a)
            h2 = R * R - (X - c[0]) ** 2 - (Y - c[1]) ** 2
            hit = h2 > 0.0
            z = np.where(hit, c[2] + np.sqrt(np.maximum(h2, 0.0)), -np.inf)
            better = z > zbest
            if better.any():
                zbest = np.where(better, z, zbest)
                idx = np.nonzero(better)[0]
                nrm[idx, 0] = (X[idx] - c[0]) / R
                nrm[idx, 1] = (Y[idx] - c[1]) / R
                nrm[idx, 2] = (z[idx] - c[2]) / R
    points = np.stack([X, Y, zbest], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    albedo = rng.uniform(0.2, 0.9, size=(P, 3))
    light = sh_lighting(rng, n_bands)
    return dict(points=_f32(points), normals=_f32(nrm), albedo=_f32(albedo),
                centers=_f32(centers), radii=_f32(radii), light=_f32(light),
                n_bands=n_bands)


def height_field_scene(seed=3, res=1024, n_spheres=300, n_bands=8, n_bumps=16):
    """Height field z = h(x, y) over [-1,1]^2 on a ``res`` x ``res`` grid, h a
    sum of ``n_bumps`` random Gaussian bumps, analytic unit normals; spheres
    hover over the field at h + U[0.05, 0.8] with radii log-uniform in
    [0.01, 0.2]; albedo uniform in [0.2, 0.9]; lighting N(0,0.3)/(l+1) with
    l=0 term 1.0."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(-0.25, 0.25, n_bumps)
    mu = rng.uniform(-1.0, 1.0, (n_bumps, 2))
    sig = rng.uniform(0.1, 0.4, n_bumps)

    def h_and_grad(x, y):
        h = np.zeros_like(x)
        hx = np.zeros_like(x)
        hy = np.zeros_like(x)
        for a, (mx, my), s in zip(amp, mu, sig):
            g = a * np.exp(-((x - mx) ** 2 + (y - my) ** 2) / (2 * s * s))
            h += g
            hx += -g * (x - mx) / (s * s)
            hy += -g * (y - my) / (s * s)
        return h, hx, hy

    t = -1.0 + (2.0 * np.arange(res) + 1.0) / res
    X, Y = np.meshgrid(t, t, indexing="xy")
    X = X.ravel()
    Y = Y.ravel()
    H, HX, HY = h_and_grad(X, Y)
    points = np.stack([X, Y, H], axis=1)
    nrm = np.stack([-HX, -HY, np.ones_like(H)], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    albedo = rng.uniform(0.2, 0.9, size=(X.size, 3))
    cxy = rng.uniform(-1.0, 1.0, (n_spheres, 2))
    ch, _, _ = h_and_grad(cxy[:, 0], cxy[:, 1])
    cz = ch + rng.uniform(0.05, 0.8, n_spheres)
    centers = np.concatenate([cxy, cz[:, None]], axis=1)
    radii = np.exp(rng.uniform(np.log(0.01), np.log(0.2), n_spheres))
    light = sh_lighting(rng, n_bands, band_decay=True)
    return dict(points=_f32(points), normals=_f32(nrm), albedo=_f32(albedo),
                centers=_f32(centers), radii=_f32(radii), light=_f32(light),
                n_bands=n_bands)


def random_scene(seed, n_points, n_spheres, n_bands, box=1.0, r_range=(0.03, 0.25),
                 inside_fraction=0.0):
    """Points uniform in a cube of half-width ``box`` with random unit normals,
    spheres uniform in the same cube.  ``inside_fraction`` of the points are
    moved inside a random sphere (the clamped, point-inside-sphere case)."""
    rng = np.random.default_rng(seed)
    points = rng.uniform(-box, box, (n_points, 3))
    normals = rng.normal(size=(n_points, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    albedo = rng.uniform(0.2, 0.9, (n_points, 3))
    centers = rng.uniform(-box, box, (n_spheres, 3))
    radii = rng.uniform(*r_range, n_spheres)
    if n_spheres > 0 and inside_fraction > 0:
        m = rng.random(n_points) < inside_fraction
        j = rng.integers(0, n_spheres, n_points)
        d = rng.normal(size=(n_points, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        q = centers[j] + d * (radii[j] * rng.uniform(0.0, 0.9, n_points))[:, None]
        points = np.where(m[:, None], q, points)
    light = sh_lighting(rng, n_bands)
    return dict(points=_f32(points), normals=_f32(normals), albedo=_f32(albedo),
                centers=_f32(centers), radii=_f32(radii), light=_f32(light),
                n_bands=n_bands)


def perturb_scene(scene, seed, center_sigma=0.01, light_sigma=0.05,
                  albedo_range=(0.9, 1.1)):
    """Copy of ``scene`` with centres + N(0, center_sigma), lighting +
    N(0, light_sigma) and albedo scaled by U[albedo_range]: the target of the
    L2 analysis-by-synthesis loss."""
    rng = np.random.default_rng(seed)
    out = dict(scene)
    out["centers"] = _f32(scene["centers"].astype(np.float64)
                          + rng.normal(0, center_sigma, scene["centers"].shape))
    out["light"] = _f32(scene["light"].astype(np.float64)
                        + rng.normal(0, light_sigma, scene["light"].shape))
    out["albedo"] = _f32(scene["albedo"].astype(np.float64)
                         * rng.uniform(*albedo_range, scene["albedo"].shape))
    return out


def serving_job(seed, n_points, n_spheres, n_bands, n_bumps=4):
    """A job of the serving mix: the first ``n_points`` samples of a square
    height-field grid (``n_bumps`` Gaussian bumps over [-1,1]^2) with analytic
    unit normals, albedo uniform in [0.2, 0.9], spheres hovering over the field
    (height + U[0.05, 0.8], radii log-uniform in [0.01, 0.2]) and lighting
    N(0,0.3)/(l+1) with l=0 term 1.0."""
    rng = np.random.default_rng(seed)
    res = int(np.ceil(np.sqrt(n_points)))
    amp = rng.uniform(-0.25, 0.25, n_bumps)
    mu = rng.uniform(-1.0, 1.0, (n_bumps, 2))
    sig = rng.uniform(0.15, 0.4, n_bumps)
    t = -1.0 + (2.0 * np.arange(res) + 1.0) / res
    X, Y = np.meshgrid(t, t, indexing="xy")
    X = X.ravel()[:n_points]
    Y = Y.ravel()[:n_points]

    def h_and_grad(x, y):
        h = np.zeros_like(x)
        hx = np.zeros_like(x)
        hy = np.zeros_like(x)
        for a, (mx, my), s in zip(amp, mu, sig):
            g = a * np.exp(-((x - mx) ** 2 + (y - my) ** 2) / (2 * s * s))
            h += g
            hx -= g * (x - mx) / (s * s)
            hy -= g * (y - my) / (s * s)
        return h, hx, hy

    H, HX, HY = h_and_grad(X, Y)
    nrm = np.stack([-HX, -HY, np.ones_like(H)], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    albedo = rng.uniform(0.2, 0.9, size=(n_points, 3))
    cxy = rng.uniform(-1.0, 1.0, (n_spheres, 2))
    ch, _, _ = h_and_grad(cxy[:, 0], cxy[:, 1])
    centers = np.concatenate([cxy, (ch + rng.uniform(0.05, 0.8, n_spheres))[:, None]], axis=1)
    radii = np.exp(rng.uniform(np.log(0.01), np.log(0.2), n_spheres))
    light = sh_lighting(rng, n_bands, band_decay=True)
    return dict(points=_f32(np.stack([X, Y, H], axis=1)), normals=_f32(nrm), albedo=_f32(albedo),
                centers=_f32(centers), radii=_f32(radii), light=_f32(light), n_bands=n_bands)


def mesh_deformation_scene(seed=2, n_theta=250, n_phi=200, n_spheres=200, n_params=60, n_views=16,
                           n_bands=4):
    """Mesh-deformation batch: a UV-sphere mesh of n_theta x n_phi vertices
    (radius 1 with a random smooth radial deformation), per-vertex normals and
    albedo; n_spheres occluder spheres inside the mesh (centres at radius
    0.5-0.8, radii U[0.05, 0.15]); vertices, normals and centres affine in
    n_params deformation parameters (basis entries N(0, 0.01)); n_views rigid
    poses (axis-angle |w| <= pi, translation N(0, 0.1)).  Returns float32
    arrays: v0, n0, A_v [M,3,D], A_n [M,3,D], c0, A_c [N,3,D], radii, albedo,
    light, poses [V,6]."""
    rng = np.random.default_rng(seed)
    th = (np.arange(n_theta) + 0.5) / n_theta * np.pi
    ph = np.arange(n_phi) / n_phi * 2 * np.pi
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    TH = TH.ravel()
    PH = PH.ravel()
    coef = rng.normal(0.0, 0.03, (4, 4))

    def radius(t, p):
        r = np.ones_like(t)
        dr_t = np.zeros_like(t)
        dr_p = np.zeros_like(t)
        for a in range(4):
            for b in range(4):
                c = coef[a, b]
                r += c * np.cos((a + 1) * t) * np.cos(b * p)
                dr_t += -c * (a + 1) * np.sin((a + 1) * t) * np.cos(b * p)
                dr_p += -c * b * np.cos((a + 1) * t) * np.sin(b * p)
        return r, dr_t, dr_p

    r, r_t, r_p = radius(TH, PH)
    u = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], axis=1)
    u_t = np.stack([np.cos(TH) * np.cos(PH), np.cos(TH) * np.sin(PH), -np.sin(TH)], axis=1)
    u_p = np.stack([-np.sin(TH) * np.sin(PH), np.sin(TH) * np.cos(PH), np.zeros_like(TH)], axis=1)
    v0 = r[:, None] * u
    e_t = r_t[:, None] * u + r[:, None] * u_t
    e_p = r_p[:, None] * u + r[:, None] * u_p
    n0 = np.cross(e_t, e_p)
    bad = np.linalg.norm(n0, axis=1) < 1e-9
    n0[bad] = u[bad]
    n0 /= np.linalg.norm(n0, axis=1, keepdims=True)
    n0 *= np.sign(np.sum(n0 * u, axis=1, keepdims=True))
    M = v0.shape[0]
    A_v = rng.normal(0.0, 0.01, (M, 3, n_params))
    A_n = rng.normal(0.0, 0.01, (M, 3, n_params))
    albedo = rng.uniform(0.2, 0.9, (M, 3))
    d = rng.normal(size=(n_spheres, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    c0 = d * rng.uniform(0.5, 0.8, (n_spheres, 1))
    A_c = rng.normal(0.0, 0.01, (n_spheres, 3, n_params))
    radii = rng.uniform(0.05, 0.15, n_spheres)
    light = sh_lighting(rng, n_bands)
    axes = rng.normal(size=(n_views, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    w = axes * rng.uniform(0.0, np.pi, (n_views, 1))
    t = rng.normal(0.0, 0.1, (n_views, 3))
    return dict(v0=_f32(v0), n0=_f32(n0), A_v=_f32(A_v), A_n=_f32(A_n), c0=_f32(c0), A_c=_f32(A_c),
                radii=_f32(radii), albedo=_f32(albedo), light=_f32(light),
                poses=_f32(np.concatenate([w, t], axis=1)), n_bands=n_bands)


def environment_map(seed=5, height=1024, width=2048, n_suns=2):
    """Equirectangular HDR radiance map [height, width, 3] (row r: polar
    angles [r, r+1] pi / height from +z; column c: azimuths [c, c+1] 2 pi /
    width), standing in for the paper's HDR environment maps: a sky whose
    colour varies with elevation, a darker ground below the horizon, ``n_suns``
    small bright discs (radiance 20-60, angular radius 2-5 degrees) and
    multiplicative 5 % noise.  All values are positive."""
    rng = np.random.default_rng(seed)
    theta = (np.arange(height) + 0.5) * np.pi / height
    phi = (np.arange(width) + 0.5) * 2.0 * np.pi / width
    st, ct = np.sin(theta)[:, None], np.cos(theta)[:, None]
    d = np.stack([st * np.cos(phi)[None, :], st * np.sin(phi)[None, :], np.broadcast_to(ct, (height, width))], -1)
    zenith = rng.uniform(0.3, 0.6, 3)
    horizon = rng.uniform(0.7, 1.0, 3)
    ground = rng.uniform(0.1, 0.3, 3)
    up = np.clip(d[..., 2:3], 0.0, 1.0)
    sky = horizon[None, None] + (zenith - horizon)[None, None] * up
    env = np.where(d[..., 2:3] >= 0.0, sky, ground[None, None])
    for _ in range(n_suns):
        el = rng.uniform(0.1, 1.3)
        az = rng.uniform(0.0, 2.0 * np.pi)
        s = np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        radius = np.deg2rad(rng.uniform(2.0, 5.0))
        disc = (d @ s) >= np.cos(radius)
        env = env + disc[..., None] * rng.uniform(20.0, 60.0) * rng.uniform(0.8, 1.0, 3)[None, None]
    env = env * rng.uniform(0.95, 1.05, size=env.shape)
    return _f32(env)


def uv_grid_faces(n_theta, n_phi):
    """Triangles [F, 3] int32 of the n_theta x n_phi vertex grid of
    mesh_deformation_scene (vertex index t * n_phi + p): two per grid cell,
    wrapping around in phi, none across the poles."""
    f = []
    for t in range(n_theta - 1):
        for p in range(n_phi):
            a, b = t * n_phi + p, t * n_phi + (p + 1) % n_phi
            c, d = a + n_phi, b + n_phi
            f.append((a, c, b))
            f.append((b, c, d))
    return np.asarray(f, dtype=np.int32)


def look_at_perspective(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), fov_deg=45.0, aspect=1.0,
                        near=0.1, far=20.0):
    """Row-major 4x4 matrix taking world [x, y, z, 1] to clip coordinates: a
    camera at ``eye`` looking at ``target`` (OpenGL-style perspective, visible
    depth mapped to NDC z in [-1, 1])."""
    eye, target, up = (np.asarray(v, np.float64) for v in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    s_ = np.cross(f, up)
    s_ /= np.linalg.norm(s_)
    u = np.cross(s_, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = s_, u, -f
    view[:3, 3] = -view[:3, :3] @ eye
    t = 1.0 / np.tan(np.deg2rad(fov_deg) / 2)
    proj = np.array([[t / aspect, 0, 0, 0], [0, t, 0, 0],
                     [0, 0, (far + near) / (near - far), 2 * far * near / (near - far)], [0, 0, -1, 0]])
    return _f32(proj @ view)
