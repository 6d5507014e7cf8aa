"""Pins of the rasterisation oracle (oracle/raster_oracle.py) against closed
forms: pixel coverage of an axis-aligned rectangle, depth order, exact affine
interpolation under an orthographic camera, perspective-correct interpolation
against ray-plane intersection, culling rules, and the adjoint against
central differences."""

import numpy as np

from oracle import raster_oracle as R


def _quad(x0, x1, y0, y1, z=0.0):
    v = np.array([[x0, y0, z], [x1, y0, z], [x1, y1, z], [x0, y1, z]], float)
    f = np.array([[0, 1, 2], [0, 2, 3]])
    return v, f


def test_rectangle_coverage_and_constant_colour():
    """A rectangle whose edges lie on pixel boundaries covers exactly the
    pixels inside it (shared diagonal counted once), in one colour."""
    H, W = 16, 24
    v, f = _quad(-0.5, 0.25, -0.75, 0.5)           # 9 x 10 pixels
    B = np.tile([0.2, 0.5, 0.9], (4, 1))
    img, fi = R.rasterize(v, f, np.eye(4), B, H, W)
    assert (fi >= 0).sum() == 9 * 10
    np.testing.assert_allclose(img[fi >= 0], np.tile([0.2, 0.5, 0.9], (90, 1)), rtol=1e-14)
    assert np.all(img[fi < 0] == 0.0)


def test_depth_order_and_tie_rule():
    """The nearer of two overlapping triangles is drawn, whatever the order."""
    v1, f1 = _quad(-1, 1, -1, 1, z=0.3)
    v2, f2 = _quad(-0.5, 0.5, -0.5, 0.5, z=-0.2)
    v = np.concatenate([v1, v2])
    B = np.concatenate([np.tile([1.0, 0, 0], (4, 1)), np.tile([0, 1.0, 0], (4, 1))])
    for faces in (np.concatenate([f1, f2 + 4]), np.concatenate([f2 + 4, f1])):
        img, fi = R.rasterize(v, faces, np.eye(4), B, 8, 8)
        assert np.all(img[2:6, 2:6] == [0, 1.0, 0]) and img[0, 0, 0] == 1.0


def test_orthographic_affine_interpolation_is_exact():
    rng = np.random.default_rng(0)
    v = np.array([[-0.9, -0.8, 0.1], [0.85, -0.6, -0.3], [0.1, 0.9, 0.5]])
    a, c0 = rng.normal(size=(3, 3)), rng.normal(size=3)
    B = v @ a + c0
    img, fi = R.rasterize(v, [[0, 1, 2]], np.eye(4), B, 20, 20)
    q = R.pixel_centres(20, 20)
    # the surface point under each pixel: (qx, qy, z) on the triangle's plane
    nrm = np.cross(v[1] - v[0], v[2] - v[0])
    z = v[0, 2] - (nrm[0] * (q[..., 0] - v[0, 0]) + nrm[1] * (q[..., 1] - v[0, 1])) / nrm[2]
    X = np.stack([q[..., 0], q[..., 1], z], -1)
    ref = X @ a + c0
    np.testing.assert_allclose(img[fi >= 0], ref[fi >= 0], atol=1e-12)


def _perspective(fov_deg=60.0, near=0.5, far=10.0):
    t = 1.0 / np.tan(np.deg2rad(fov_deg) / 2)
    return np.array([[t, 0, 0, 0], [0, t, 0, 0],
                     [0, 0, (far + near) / (near - far), 2 * far * near / (near - far)], [0, 0, -1, 0]])


def test_perspective_correct_interpolation_matches_ray_plane_intersection():
    """Under a perspective camera the colour at a pixel equals the affine
    radiance evaluated at the point where the pixel's ray meets the triangle."""
    P = _perspective()
    v = np.array([[-1.0, -0.8, -3.0], [1.2, -0.5, -5.0], [0.1, 1.0, -2.5]])
    rng = np.random.default_rng(1)
    a, c0 = rng.normal(size=(3, 3)), rng.normal(size=3)
    B = v @ a + c0
    img, fi = R.rasterize(v, [[0, 1, 2]], P, B, 24, 24)
    assert (fi >= 0).sum() > 50
    Pinv = np.linalg.inv(P)
    q = R.pixel_centres(24, 24)
    nrm = np.cross(v[1] - v[0], v[2] - v[0])
    for r, c in zip(*np.nonzero(fi >= 0)):
        # ray: world points X(z) = dehomog(Pinv [qx, qy, z, 1]); the camera sits at the origin
        h = Pinv @ np.array([q[r, c, 0], q[r, c, 1], 0.0, 1.0])
        d = h[:3] / h[3]                            # a point on the ray through the origin
        t = np.dot(nrm, v[0]) / np.dot(nrm, d)
        X = t * d
        np.testing.assert_allclose(img[r, c], X @ a + c0, atol=1e-10)


def test_culling_rules():
    """Triangles with a vertex behind the camera (w <= 0) or outside the depth
    range are not drawn."""
    P = _perspective()
    v = np.array([[-1.0, -1.0, -3.0], [1.0, -1.0, -3.0], [0.0, 1.0, 1.0]])   # third vertex behind
    img, fi = R.rasterize(v, [[0, 1, 2]], P, np.ones((3, 3)), 8, 8)
    assert np.all(fi == -1)
    v2, f2 = _quad(-1, 1, -1, 1, z=1.5)
    img, fi = R.rasterize(v2, f2, np.eye(4), np.ones((4, 3)), 8, 8)
    assert np.all(fi == -1)


def test_adjoint_matches_central_differences():
    P = _perspective()
    rng = np.random.default_rng(2)
    v = np.array([[-1.0, -0.8, -3.0], [1.2, -0.5, -5.0], [0.1, 1.0, -2.5], [1.3, 1.1, -4.0]])
    faces = np.array([[0, 1, 2], [1, 3, 2]])
    B = rng.uniform(0.1, 1.0, size=(4, 3))
    img, fi = R.rasterize(v, faces, P, B, 20, 20)
    dI = rng.normal(size=img.shape)
    g = R.rasterize_backward(v, faces, P, B, fi, dI)
    h = 1e-6
    for name, base, grad in (("radiance", B, g["d_radiance"]), ("vertices", v, g["d_vertices"])):
        for idx in np.ndindex(base.shape):
            p, m = base.copy(), base.copy()
            p[idx] += h
            m[idx] -= h
            args_p = (p, faces, P, B) if name == "vertices" else (v, faces, P, p)
            args_m = (m, faces, P, B) if name == "vertices" else (v, faces, P, m)
            fd = np.sum(dI * (R.shade_pixels(*args_p, fi) - R.shade_pixels(*args_m, fi))) / (2 * h)
            assert abs(fd - grad[idx]) < 1e-6 * max(1.0, abs(fd)), (name, idx, fd, grad[idx])
