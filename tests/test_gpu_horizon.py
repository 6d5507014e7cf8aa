"""Horizon culling (configuration horizon_cull = 1): per point, a sphere lying
entirely below the tangent plane, (c - x) . n_hat < -r, is left out.  The CUDA
library is compared with the FP64 oracle making the same selection, on points
whose every pair is clear of the selection boundary by a relative margin
(float32 and float64 may decide a pair on the boundary differently, and the
selection moves a whole sphere's contribution)."""

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

from gpu_helpers import FIELDS, gpu_run, grad_err, oracle_k_consistent, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4
TOL_GRAD_8 = 3e-4      # 8-band gradients (same gate as the other 8-band tests)


def _clear_scene(seed, n_points, n_spheres, n):
    sc = S.random_scene(seed, n_points, n_spheres, n, inside_fraction=0.05)
    pts = sc["points"].astype(np.float64)
    nrm = sc["normals"].astype(np.float64)
    nh = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    d = sc["centers"].astype(np.float64)[None] - pts[:, None]
    margin = np.einsum("pjc,pc->pj", d, nh) + sc["radii"].astype(np.float64)[None]
    keep = np.all(np.abs(margin) > 1e-4 * (1.0 + np.abs(d).sum(-1)), axis=1)
    out = dict(sc)
    for k in ("points", "normals", "albedo"):
        out[k] = np.ascontiguousarray(sc[k][keep])
    culled = (margin[keep] < 0).mean()
    assert 0.1 < culled < 0.9, culled                  # the selection is exercised both ways
    return out


@pytest.mark.parametrize("n", [2, 4, 5, 6, 8])
def test_forward_with_horizon_cull(n):
    sc = _clear_scene(400 + n, 500, 37, n)
    cfg = O.Config(n_bands=n, horizon_cull=True)
    B, k, f, _, status = gpu_run(sc, cfg)
    assert status == 0
    ref = O.shade_forward(cfg, *[sc[x] for x in FIELDS], k=k)
    oracle_k_consistent(cfg, O.shade_forward(cfg, *[sc[x] for x in FIELDS])["f"], k)
    np.testing.assert_allclose(f, ref["f"], rtol=0, atol=2e-5 * max(1.0, np.abs(ref["f"]).max()))
    assert rel_err(B, ref["radiance"]).max() <= TOL
    # culling changes the answer on this scene
    B_all, *_ = gpu_run(sc, O.Config(n_bands=n))
    assert rel_err(B_all, ref["radiance"]).max() > 1e-2


@pytest.mark.parametrize("n,n_spheres,saved", [(4, 9, True), (4, 40, True), (4, 40, False), (3, 33, True),
                                               (6, 12, True), (8, 10, True)])
def test_backward_with_horizon_cull(n, n_spheres, saved):
    sc = _clear_scene(500 + n + n_spheres, 300, n_spheres, n)
    cfg = O.Config(n_bands=n, horizon_cull=True)
    dB = np.random.default_rng(6).normal(size=sc["points"].shape).astype(np.float32)
    B, k, f, g, status = gpu_run(sc, cfg, dB=dB, saved=saved)
    assert status == 0
    ref = O.shade_backward(cfg, *[sc[x] for x in FIELDS], dB, k=k)
    tol = TOL_GRAD_8 if n == 8 else TOL
    for name in ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals"):
        err = grad_err(name, g[name], ref)
        assert err.max() <= tol, f"{name}: max err {err.max():.3e}"


def test_horizon_cull_is_a_no_op_when_every_sphere_is_above():
    """The 32x32 plane: normals +z and every sphere above z = 0, so no pair is
    culled and both settings give the same shading and gradients."""
    sc = S.plane_grid_scene(seed=0)
    dB = np.random.default_rng(8).normal(size=sc["points"].shape).astype(np.float32)
    B0, _, _, g0, _ = gpu_run(sc, O.Config(n_bands=4), dB=dB)
    B1, _, _, g1, _ = gpu_run(sc, O.Config(n_bands=4, horizon_cull=True), dB=dB)
    np.testing.assert_allclose(B1, B0, rtol=1e-6, atol=1e-7 * np.abs(B0).max())
    for name in g0:
        np.testing.assert_allclose(g1[name], g0[name], rtol=1e-6, atol=1e-6 * np.abs(g0[name]).max())
