"""CUDA library vs the FP64 oracle, element by element, on seeded inputs.

Tolerance (FP32 path): the normalised error |x - x_ref| / max(|x_ref|,
1e-3 max|x_ref|) must stay <= 1e-4 for the radiance and for every gradient
output; for the gradient sums over points (lighting, centres, radii) the scale
also includes 1e-2 x the sum of absolute per-point terms (see grad_err).  Per-point squaring counts k are compared exactly; a point whose k
differs must lie on a boundary |f_hat| = tau 2^k (float32 vs float64 tie), and
the oracle is then evaluated with the GPU's k for that point."""

import numpy as np
import pytest

from oracle import shs_oracle as O
from paper_2104_00359_gb300 import synthetic as S

from gpu_helpers import FIELDS, gpu_run, grad_err, oracle_k_consistent, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-4
TOL_GRAD_8 = 3e-4


def _oracle_forward(sc, cfg, k):
    return O.shade_forward(cfg, *[sc[f] for f in FIELDS], k=k)


def _check_forward(sc, cfg, tol=TOL):
    B, k, f, _, status = gpu_run(sc, cfg)
    assert status == 0
    ref = _oracle_forward(sc, cfg, k)
    np.testing.assert_allclose(f, ref["f"], rtol=0, atol=2e-5 * max(1.0, np.abs(ref["f"]).max()))
    if cfg.fixed_k < 0:
        oracle_k_consistent(cfg, ref["f"], k)
    err = rel_err(B, ref["radiance"])
    assert err.max() <= tol, f"radiance max err {err.max():.3e}"
    return B, k


def test_forward_plane_grid_32x32():
    """32x32 plane, 8 spheres, n=4 (some points inside spheres)."""
    _check_forward(S.plane_grid_scene(seed=0), O.Config(n_bands=4))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_forward_random_all_band_counts(n):
    """Several 128-point tiles plus a ragged tail (P = 421), 13 spheres, some
    points inside spheres."""
    sc = S.random_scene(100 + n, 421, 13, n, inside_fraction=0.1)
    _check_forward(sc, O.Config(n_bands=n))


def test_forward_fixed_k_and_tau():
    sc = S.random_scene(7, 300, 10, 4)
    _check_forward(sc, O.Config(n_bands=4, fixed_k=5))
    _check_forward(sc, O.Config(n_bands=4, exp_tau=0.25, exp_kmax=6))


def test_forward_no_spheres_closed_form():
    sc = S.random_scene(8, 200, 0, 4)
    B, _ = _check_forward(sc, O.Config(n_bands=4))
    from scipy.special import sph_harm_y  # noqa: F401  (closed form via the oracle pin)
    Ahat = np.array([np.pi, 2 * np.pi / 3, np.pi / 4, 0.0])[O.band_of(16)]
    nrm = sc["normals"].astype(np.float64)
    Y = O.real_sh(4, nrm / np.linalg.norm(nrm, axis=1, keepdims=True))
    ref = sc["albedo"] * ((Y * Ahat) @ sc["light"].astype(np.float64).T)
    assert rel_err(B, ref).max() <= TOL


def test_point_at_sphere_centre_and_inside():
    sc = S.random_scene(9, 130, 4, 4)
    sc["points"][0] = sc["centers"][0]              # D = 0: sphere skipped
    sc["points"][1] = sc["centers"][1] + 0.1 * sc["radii"][1]   # inside: hemisphere cap
    _check_forward(sc, O.Config(n_bands=4))


def test_zero_points():
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    sc = S.random_scene(10, 5, 3, 4)
    dev = torch.device("cuda:0")
    scene = Scene(torch.from_numpy(sc["centers"]).to(dev), torch.from_numpy(sc["radii"]).to(dev),
                  torch.from_numpy(sc["light"]).to(dev), Config())
    e = torch.empty((0, 3), device=dev)
    B = scene.shade(e, e, e)
    g = scene.backward(e, e, e, e)
    torch.cuda.synchronize()
    assert B.shape == (0, 3)
    assert float(g["d_light"].abs().sum()) == 0.0 and float(g["d_centers"].abs().sum()) == 0.0
    scene.close()


# --------------------------------------------------------------------------- backward

def _check_backward(sc, cfg, saved=True, tol=TOL, want=None):
    rng = np.random.default_rng(5)
    dB = rng.normal(size=sc["points"].shape).astype(np.float32)
    B, k, f, g, status = gpu_run(sc, cfg, dB=dB, saved=saved, want=want)
    assert status == 0
    ref = O.shade_backward(cfg, *[sc[x] for x in FIELDS], dB, k=k)
    for name in ref:
        if name not in g or g[name] is None:
            continue
        err = grad_err(name, g[name], ref)
        assert err.max() <= tol, f"{name}: max err {err.max():.3e} at {np.unravel_index(err.argmax(), err.shape)}"
    return g, ref


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_backward_all_gradients(n):
    """Every gradient output against the oracle, horizon culling off.  From 7
    bands the triple products run through the quadrature and the adjoint runs
    back through the k squarings, each doubling the relative rounding of its
    operand: gradients there are gated at 3e-4 (the radiance stays at 1e-4)."""
    sc = S.random_scene(200 + n, 300, 9, n, inside_fraction=0.1)
    _check_backward(sc, O.Config(n_bands=n), tol=TOL if n <= 6 else TOL_GRAD_8)


@pytest.mark.parametrize("n", [7, 8])
def test_backward_all_gradients_recompute(n):
    """As above with saved = NULL: the split backward recomputes f."""
    sc = S.random_scene(210 + n, 260, 11, n, inside_fraction=0.1)
    _check_backward(sc, O.Config(n_bands=n), saved=False, tol=TOL_GRAD_8)


def test_backward_plane_grid():
    _check_backward(S.plane_grid_scene(seed=0), O.Config(n_bands=4))


def test_backward_recompute_equals_saved():
    sc = S.random_scene(11, 260, 7, 4)
    g1, _ = _check_backward(sc, O.Config(n_bands=4), saved=True)
    g2, _ = _check_backward(sc, O.Config(n_bands=4), saved=False)
    for name in g1:
        np.testing.assert_allclose(g1[name], g2[name], rtol=1e-6, atol=1e-6 * np.abs(g1[name]).max())


def test_backward_subset_of_outputs():
    sc = S.random_scene(12, 200, 6, 4)
    g, _ = _check_backward(sc, O.Config(n_bands=4), want=("light", "radii"))
    assert g["d_albedo"] is None and g["d_points"] is None and g["d_centers"] is None


def test_backward_l2_loss():
    sc = S.random_scene(13, 333, 8, 4)
    tgt = S.perturb_scene(sc, 1)
    cfg = O.Config(n_bands=4)
    target = O.shade_forward(cfg, *[tgt[x] for x in FIELDS])["radiance"].astype(np.float32)
    B, k, f, g, status = gpu_run(sc, cfg, l2_target=target)
    assert status == 0
    dB = B.astype(np.float64) - target
    ref = O.shade_backward(cfg, *[sc[x] for x in FIELDS], dB, k=k)
    loss_ref = 0.5 * np.sum(dB ** 2)
    assert abs(float(g["loss"]) - loss_ref) <= 1e-5 * loss_ref
    for name in ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals"):
        assert grad_err(name, g[name], ref).max() <= TOL, name


def test_atomic_and_deterministic_modes_agree():
    sc = S.random_scene(14, 1000, 12, 4)
    cfg_d = O.Config(n_bands=4)
    cfg_a = O.Config(n_bands=4)
    cfg_a.deterministic = False
    dB = np.random.default_rng(3).normal(size=sc["points"].shape).astype(np.float32)
    _, k, _, gd, _ = gpu_run(sc, cfg_d, dB=dB)
    _, _, _, gd2, _ = gpu_run(sc, cfg_d, dB=dB)
    _, _, _, ga, _ = gpu_run(sc, cfg_a, dB=dB)
    ref = O.shade_backward(cfg_d, *[sc[x] for x in FIELDS], dB, k=k)
    for name in ("d_light", "d_centers", "d_radii"):
        assert np.array_equal(gd[name], gd2[name]), name     # fixed reduction order
        assert grad_err(name, ga[name], ref).max() <= TOL, name
        assert grad_err(name, gd[name], ref).max() <= TOL, name


def test_autograd_function_matches_direct_backward():
    import torch
    from paper_2104_00359_gb300 import Config, Scene, shade
    sc = S.random_scene(15, 257, 6, 4)
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(sc[k]).to(dev).requires_grad_(True) for k in FIELDS}
    scene = Scene(T["centers"].detach(), T["radii"].detach(), T["light"].detach(), Config())
    B = shade(T["points"], T["normals"], T["albedo"], T["centers"], T["radii"], T["light"], scene)
    dB = torch.from_numpy(np.random.default_rng(16).normal(size=tuple(B.shape)).astype(np.float32)).to(dev)
    B.backward(dB)
    sv = scene.new_saved(B.shape[0], dev)
    scene.shade(T["points"].detach(), T["normals"].detach(), T["albedo"].detach(), saved=sv)
    k = scene.saved_views(sv, B.shape[0])[1].cpu().numpy().astype(np.int64)
    ref = O.shade_backward(O.Config(n_bands=4), *[sc[x] for x in FIELDS], dB.cpu().numpy(), k=k)
    name_map = dict(points="d_points", normals="d_normals", albedo="d_albedo", centers="d_centers",
                    radii="d_radii", light="d_light")
    for k_, t in T.items():
        assert grad_err(name_map[k_], t.grad.cpu().numpy(), ref).max() <= TOL, k_
    scene.close()


@pytest.mark.parametrize("n,prec", [(4, 0), (6, 0), (8, 0), (8, 2), (8, 1)])
def test_shade_tail_after_lighting_update(n, prec):
    """shs_shade_tail: with the saved log-visibility of an earlier shs_shade
    and new lighting, only the exponential and Eq. 8 run; the radiance equals
    a full forward with the new lighting (FP32: bitwise) and the oracle."""
    import torch
    from paper_2104_00359_gb300 import Config, Scene
    sc = S.random_scene(400 + n + prec, 333, 11, n, inside_fraction=0.05)
    dev = torch.device("cuda:0")
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in FIELDS}
    P = sc["points"].shape[0]
    scene = Scene(T["centers"], T["radii"], T["light"], Config(n_bands=n, precision=prec))
    sv = scene.new_saved(P, dev)
    scene.shade(T["points"], T["normals"], T["albedo"], saved=sv)
    light2 = np.random.default_rng(9).normal(scale=0.3, size=sc["light"].shape).astype(np.float32)
    light2[:, 0] = 1.0
    alb2 = np.ascontiguousarray(sc["albedo"][::-1], np.float32)
    scene.update(light=torch.from_numpy(light2).to(dev))
    Bt = scene.shade_tail(T["normals"], torch.from_numpy(alb2).to(dev), sv)
    Bf = scene.shade(T["points"], T["normals"], torch.from_numpy(alb2).to(dev))
    torch.cuda.synchronize()
    assert scene.device_status() == 0
    k = scene.saved_views(sv, P)[1].cpu().numpy().astype(np.int64)
    scene.close()
    if prec == 0:
        np.testing.assert_array_equal(Bt.cpu().numpy(), Bf.cpu().numpy())
    sc2 = dict(sc, light=light2, albedo=alb2)
    ref = O.shade_forward(O.Config(n_bands=n), *[sc2[f] for f in FIELDS], k=k)["radiance"]
    assert rel_err(Bt.cpu().numpy(), ref).max() <= (TOL if prec == 0 else 2e-3)
