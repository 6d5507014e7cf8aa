"""Eq. 9 projection of an equirectangular map onto SH lighting: the CUDA
kernel (shs_project_envmap) against the FP64 oracle's pixel sum.

Each coefficient is a sum over all pixels of terms of either sign, so the
gate scale includes 1e-2 x the sum of the absolute terms (float32
accumulation in any order is accurate to a few ulps of that sum), as for the
other summed outputs."""

import math

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _abs_terms(n, env):
    """sum over pixels of |value| |y_i| d_omega, [3, K]."""
    env = np.abs(np.asarray(env, np.float64))
    H, W = env.shape[:2]
    dirs, d_omega = O.envmap_directions(H, W)
    out = np.zeros((3, n * n))
    step = max(1, 65536 // W)
    for r0 in range(0, H, step):
        Y = np.abs(O.real_sh(n, dirs[r0:r0 + step]))
        out += np.einsum("hwc,hwk->ck", env[r0:r0 + step] * d_omega[r0:r0 + step, None, None], Y)
    return out


def _gpu(env, n):
    import torch
    from paper_2104_00359_gb300.envmap import project_envmap
    t = torch.from_numpy(np.ascontiguousarray(env)).cuda()
    L = project_envmap(t, n)
    torch.cuda.synchronize()
    return L.cpu().numpy()


def _check(env, n, tol=TOL):
    got = _gpu(env, n)
    ref = O.project_envmap(n, env)
    a = _abs_terms(n, env)
    scale = np.maximum(np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max()), 1e-2 * a)
    err = np.abs(got - ref) / scale
    assert err.max() <= tol, f"n={n} {env.shape}: max err {err.max():.3e}"
    return got, ref


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_envmap_small_all_band_counts(n):
    _check(S.environment_map(seed=10 + n, height=48, width=96), n)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (37, 50), (5, 129), (300, 2), (20, 36), (3, 16), (9, 80), (2, 16400)])
def test_envmap_ragged_and_degenerate_shapes(shape):
    """Widths that take each load path: scalar (odd), float4 rows (width a
    multiple of 4) and the four-fold symmetry path (a multiple of 16)."""
    rng = np.random.default_rng(sum(shape))
    env = rng.uniform(0.0, 2.0, size=shape + (3,)).astype(np.float32)
    _check(env, 4)
    _check(env, 8)


def test_envmap_unaligned_map_pointer():
    """A map that starts 4 bytes into its allocation (not 16-byte aligned)
    takes the scalar-load path and gives the same result."""
    import torch
    from paper_2104_00359_gb300.envmap import project_envmap
    env = S.environment_map(seed=12, height=40, width=64)
    buf = torch.zeros(env.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(env.ravel()).cuda()
    view = buf[1:].view(40, 64, 3)
    assert view.data_ptr() % 16 != 0
    got = project_envmap(view, 6).cpu().numpy()
    ref = _gpu(env, 6)
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def test_envmap_constant_map_dc():
    """A constant map gives L_0 = c sqrt(4 pi) (the pixel solid angles tile
    the sphere) and vanishing m != 0 coefficients."""
    env = np.full((64, 128, 3), 1.5, np.float32)
    got = _gpu(env, 4)
    np.testing.assert_allclose(got[:, 0], 1.5 * math.sqrt(4 * math.pi), rtol=2e-6)
    m = np.array([mm for l in range(4) for mm in range(-l, l + 1)])
    assert np.abs(got[:, m != 0]).max() < 1e-5


def test_envmap_full_size_1024x2048_n8_and_deterministic():
    import torch
    from paper_2104_00359_gb300.envmap import project_envmap
    env = S.environment_map(seed=5, height=1024, width=2048)
    got, _ = _check(env, 8)
    t = torch.from_numpy(env).cuda()
    again = project_envmap(t, 8).cpu().numpy()
    assert np.array_equal(got, again)


def test_envmap_lighting_feeds_a_scene():
    """The projected lighting drives the shading path: with no spheres the
    radiance of a projected clamped-cosine-weighted map matches the oracle
    shading with the oracle's projection."""
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    from paper_2104_00359_gb300.envmap import project_envmap
    env = S.environment_map(seed=6, height=128, width=256)
    light = project_envmap(torch.from_numpy(env).cuda(), 4)
    sc = S.random_scene(7, 200, 0, 4)
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in ("points", "normals", "albedo")}
    scene = Scene(None, None, light, Config(n_bands=4))
    B = scene.shade(T["points"], T["normals"], T["albedo"]).cpu().numpy()
    scene.close()
    ref = O.shade_forward(O.Config(n_bands=4), sc["points"], sc["normals"], sc["albedo"], np.zeros((0, 3)),
                          np.zeros(0), O.project_envmap(4, env))["radiance"]
    err = np.abs(B - ref) / np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    assert err.max() <= 2e-4, err.max()
